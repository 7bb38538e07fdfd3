"""Learned cost model and autotuner for TOCAB PageRank (host orchestration; the network's
forward/backward/Adam and the feature extraction run in libtocab's CUDA kernels).

The model maps 16 features of a graph (tc_graph_features) or of a TOCAB subgraph
(tc_part_features) to five choices: for PageRank the block count (the paper's block-size
trade-off, Sec. 4.3), the load-balancing variant of the unstaged gather (Sec. 3.2) and the
direction (pull or push, Sec. 3.1); for BFS the frontier fraction above which a level runs
blocked (TOCAB's working-set threshold, Sec. 3.3) and the one below which it runs top-down
(the push phases of push-pull-push).  The load-balancing head also runs on each subgraph's
features to pick that subgraph's variant (per_block_lb, applied with tc_part_set_lb).  It
never changes results, only the time.  Without a model the choice falls back to the paper's
heuristic: pull, W from the L2 size (Sec. 4.3, Table 3), thread/warp/CTA load balancing, and
for BFS the thresholds 0.05 and 1/24.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import statistics

import numpy as np
import torch

from . import _lib as L
from . import (TocabError, _check, _stream, graph_load_csr, pagerank_pull, pagerank_push,  # noqa: F401
               tocab_partition)

BLOCK_CLASSES = ["unblocked", 1, 2, 4, 8, 16, 32, 64, "smem"]
LB_CLASSES = ["hybrid", "serial", "warp"]      # rows >= 32 edges by warp / all lane-serial / all by warp
LB_WARP_MIN = {"hybrid": 32, "serial": 1 << 30, "warp": 1}
DIR_CLASSES = ["pull", "push"]
TAU_CLASSES = [-1.0, 0.0, 0.02, 0.05, 0.1, 0.2]  # BFS blocked levels: never, always, frontier > tau V
PUSH_CLASSES = [0.0, 1.0 / 96, 1.0 / 24, 1.0 / 6]  # BFS top-down levels: never, frontier < p V
BFS_HEURISTIC = (0.05, 1.0 / 24)
HEADS = (len(BLOCK_CLASSES), len(LB_CLASSES), len(DIR_CLASSES), len(TAU_CLASSES), len(PUSH_CLASSES))
N_FEATURES = 16
HIDDEN = 64
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.json")


def graph_features(G) -> np.ndarray:
    f = np.zeros(N_FEATURES, np.float32)
    _check(L.load().tc_graph_features(G.handle, f.ctypes.data), "tc_graph_features")
    return f


def part_features(P) -> np.ndarray:
    f = np.zeros((P.num_blocks, N_FEATURES), np.float32)
    _check(L.load().tc_part_features(P.handle, f.ctypes.data), "tc_part_features")
    return f


class MLP:
    """The cost model's network, held on the device by libtocab (tc_mlp_*)."""

    def __init__(self, n_in: int = N_FEATURES, hidden: int = HIDDEN, heads=HEADS):
        self.heads = tuple(int(h) for h in heads)
        hs = (C.c_int32 * len(self.heads))(*self.heads)
        self._h = C.c_void_p()
        _check(L.load().tc_mlp_create(n_in, hidden, len(self.heads), hs, C.byref(self._h)), "tc_mlp_create")
        self.n_in, self.hidden = n_in, hidden
        self.nparams = int(L.load().tc_mlp_num_params(self._h))
        self.mu = np.zeros(n_in, np.float32)
        self.sd = np.ones(n_in, np.float32)

    def __del__(self):
        try:
            if self._h:
                L.load().tc_mlp_free(self._h)
                self._h = None
        except Exception:
            pass

    # parameter layout: W1[in][h], b1, W2[h][h], b2, W3[h][out], b3
    def shapes(self):
        out = sum(self.heads)
        return [("W1", (self.n_in, self.hidden)), ("b1", (self.hidden,)), ("W2", (self.hidden, self.hidden)),
                ("b2", (self.hidden,)), ("W3", (self.hidden, out)), ("b3", (out,))]

    def init(self, seed: int = 0):
        rng = np.random.default_rng(seed)
        p = {}
        for name, shp in self.shapes():
            fan_in = shp[0] if len(shp) == 2 else 1
            p[name] = (rng.normal(0, np.sqrt(2.0 / fan_in), shp) if len(shp) == 2 else np.zeros(shp))
        self.set(p)

    def set(self, p: dict):
        flat = np.concatenate([np.asarray(p[n], np.float32).reshape(-1) for n, _ in self.shapes()])
        assert flat.size == self.nparams
        _check(L.load().tc_mlp_set_params(self._h, np.ascontiguousarray(flat).ctypes.data), "tc_mlp_set_params")

    def _unflat(self, flat):
        out, o = {}, 0
        for n, shp in self.shapes():
            k = int(np.prod(shp))
            out[n] = flat[o:o + k].reshape(shp).astype(np.float64)
            o += k
        return out

    def get(self) -> dict:
        flat = np.zeros(self.nparams, np.float32)
        _check(L.load().tc_mlp_get_params(self._h, flat.ctypes.data, None), "tc_mlp_get_params")
        return self._unflat(flat)

    def grads(self) -> dict:
        flat = np.zeros(self.nparams, np.float32)
        _check(L.load().tc_mlp_get_params(self._h, None, flat.ctypes.data), "tc_mlp_get_params")
        return self._unflat(flat)

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32)
        Z = np.zeros((X.shape[0], sum(self.heads)), np.float32)
        _check(L.load().tc_mlp_forward(self._h, X.ctypes.data, X.shape[0], Z.ctypes.data, L.TC_MEM_HOST,
                                       _stream()), "tc_mlp_forward")
        return Z

    def loss_grad(self, X, Y) -> float:
        X = np.ascontiguousarray(X, np.float32)
        Y = np.ascontiguousarray(Y, np.int32)
        loss = C.c_double()
        _check(L.load().tc_mlp_loss_grad(self._h, X.ctypes.data, Y.ctypes.data, X.shape[0], L.TC_MEM_HOST,
                                         C.byref(loss), _stream()), "tc_mlp_loss_grad")
        return loss.value

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        _check(L.load().tc_mlp_adam_step(self._h, lr, b1, b2, eps, _stream()), "tc_mlp_adam_step")

    def train(self, X, Y, epochs=300, batch=64, lr=3e-3, seed=0) -> float:
        """Standardise features, then minibatch Adam on the device (the order of samples is
        reshuffled with a seeded generator every call of tc_mlp_train over `epochs` chunks)."""
        X = np.asarray(X, np.float32)
        Y = np.asarray(Y, np.int32)
        self.mu = X.mean(axis=0)
        self.sd = X.std(axis=0) + 1e-6
        Xs = ((X - self.mu) / self.sd).astype(np.float32)
        rng = np.random.default_rng(seed)
        loss = C.c_double()
        rounds = 10
        for r in range(rounds):
            perm = rng.permutation(len(Xs))
            Xp = np.ascontiguousarray(Xs[perm])
            Yp = np.ascontiguousarray(Y[perm])
            _check(L.load().tc_mlp_train(self._h, Xp.ctypes.data, Yp.ctypes.data, len(Xp), max(1, epochs // rounds),
                                         batch, lr, L.TC_MEM_HOST, C.byref(loss), _stream()), "tc_mlp_train")
        return loss.value

    def predict(self, X) -> np.ndarray:
        X = (np.asarray(X, np.float32).reshape(-1, self.n_in) - self.mu) / self.sd
        Z = self.forward(X)
        out, o = [], 0
        for h in self.heads:
            out.append(Z[:, o:o + h].argmax(axis=1))
            o += h
        return np.stack(out, axis=1)

    def save(self, path=WEIGHTS, meta=None):
        p = self.get()
        d = {k: v.tolist() for k, v in p.items()}
        d.update({"mu": self.mu.tolist(), "sd": self.sd.tolist(), "heads": list(self.heads),
                  "block_classes": [str(b) for b in BLOCK_CLASSES], "lb_classes": LB_CLASSES,
                  "dir_classes": DIR_CLASSES, "tau_classes": TAU_CLASSES, "push_classes": PUSH_CLASSES,
                  "meta": meta or {}})
        with open(path, "w") as fh:
            json.dump(d, fh)

    @classmethod
    def load(cls, path=WEIGHTS):
        d = json.load(open(path))
        m = cls(heads=d["heads"])
        m.set({n: np.asarray(d[n]) for n, _ in m.shapes()})
        m.mu = np.asarray(d["mu"], np.float32)
        m.sd = np.asarray(d["sd"], np.float32)
        m.meta = d.get("meta", {})
        return m


# ------------------------------------------------------------------------------------------------
# configurations and timing
# ------------------------------------------------------------------------------------------------

def _partition(G, direction, block):
    if block == "unblocked":
        return None
    d = L.TC_PULL if direction == "pull" else L.TC_PUSH
    if block == "smem":
        if direction != "pull":
            return None
        return tocab_partition(G, d, 0, block_policy="smem")
    nb = min(int(block), G.V)
    return tocab_partition(G, d, nb, smem_stage=-1)


def time_config(G, direction: str, block, lb: str = "hybrid", iters: int = 5, reps: int = 3, part=None) -> float:
    """Device time (ms) per PageRank iteration for one configuration (median of reps)."""
    if direction == "push" and block == "smem":
        return float("inf")
    P = part if part is not None else _partition(G, direction, block)
    fn = pagerank_pull if direction == "pull" else pagerank_push
    out = torch.empty(G.V, dtype=torch.float32, device="cuda")
    kw = {"lb_warp_min": LB_WARP_MIN[lb]}
    fn(G, P, iters=iters, out=out, **kw)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn(G, P, iters=iters, out=out, **kw)
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e) / iters)
    return statistics.median(ts)


def time_bfs(G, P, tau: float, push: float, sources, reps: int = 2) -> float:
    """Device time (ms) of BFS from `sources` (summed) with these thresholds, median of reps."""
    from . import bfs_pull
    lv = torch.empty(G.V, dtype=torch.int32, device="cuda")
    bfs_pull(G, P, int(sources[0]), tocab_threshold=tau, out=lv, push_threshold=push)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        for src in sources:
            bfs_pull(G, P, int(src), tocab_threshold=tau, out=lv, push_threshold=push)
        e.record()
        e.synchronize()
        ts.append(s.elapsed_time(e))
    return statistics.median(ts)


def measure_bfs(G, sources=None, reps: int = 2):
    """BFS time of every (tau, push) class pair on the paper's L2-rule partition.  Levels that
    pull on a graph of thousands of levels rescan every unvisited vertex each time, so on graphs
    above 2^20 vertices only the direction-optimised classes (push > 0) are timed."""
    P = tocab_partition(G, L.TC_PULL, 0, block_policy="l2")
    src = sources if sources is not None else [0, G.V // 2]
    table = {}
    for ti, tau in enumerate(TAU_CLASSES):
        for pi, push in enumerate(PUSH_CLASSES):
            if push == 0.0 and G.V > (1 << 20):
                continue
            table[(ti, pi)] = time_bfs(G, P, tau, push, src, reps)
    best = min(table, key=table.get)
    return {"labels": best, "table": {f"bfs|{TAU_CLASSES[t]:g}|{PUSH_CLASSES[q]:.4g}": v
                                      for (t, q), v in table.items()}}


def heuristic_config():
    """The method without the model: pull, the paper's L2-derived block width, hybrid LB."""
    return ("pull", "l2", "hybrid")


def measure_graph(G, iters=5, reps=3, bfs_src=None):
    """Times of every (direction, block class) with hybrid LB, and of every LB variant for the
    best unstaged pull block class.  Returns dict with labels and the timing table."""
    table = {}
    for d in DIR_CLASSES:
        for b in BLOCK_CLASSES:
            if d == "push" and b == "smem":
                continue
            if not isinstance(b, str) and b > G.V:
                continue
            try:
                table[(d, str(b), "hybrid")] = time_config(G, d, b, "hybrid", iters, reps)
            except TocabError:
                pass
    best_pull_unstaged = min((t, b) for (d, b, lb), t in table.items() if d == "pull" and b != "smem")[1]
    bu = best_pull_unstaged if best_pull_unstaged == "unblocked" else int(best_pull_unstaged)
    P = _partition(G, "pull", bu)
    for lb in LB_CLASSES[1:]:
        table[("pull", str(best_pull_unstaged), lb)] = time_config(G, "pull", bu, lb, iters, reps, part=P)
    t_l2 = time_config(G, "pull", None, "hybrid", iters, reps, part=tocab_partition(G, L.TC_PULL, 0))
    table[("pull", "l2", "hybrid")] = t_l2
    best = min(table.items(), key=lambda kv: kv[1])
    bdir = best[0][0]
    pull_blocks = {b: t for (d, b, lb), t in table.items() if d == "pull" and lb == "hybrid" and b != "l2"}
    bblock = min(pull_blocks, key=pull_blocks.get)
    lbs = {lb: t for (d, b, lb), t in table.items() if d == "pull" and b == str(best_pull_unstaged)}
    blb = min(lbs, key=lbs.get)
    bfs = measure_bfs(G, bfs_src)
    labels = (BLOCK_CLASSES.index(bblock if bblock in ("unblocked", "smem") else int(bblock)),
              LB_CLASSES.index(blb), DIR_CLASSES.index(bdir)) + tuple(bfs["labels"])
    out = {"|".join(map(str, k)): v for k, v in table.items()}
    out.update(bfs["table"])
    return {"labels": labels, "table": out}


def choose(model, G, P_probe=None):
    """The model's PageRank configuration for graph G: (direction, block class, LB variant)."""
    f = graph_features(G)
    blk_c, lb_c, dir_c = model.predict(f[None])[0][:3]
    direction = DIR_CLASSES[dir_c]
    block = BLOCK_CLASSES[blk_c]
    lb = LB_CLASSES[lb_c]
    if direction == "push" and block == "smem":
        block = 64
    return direction, block, lb


def choose_bfs(model, G):
    """The model's BFS thresholds for graph G: (tocab_threshold, push_threshold)."""
    pred = model.predict(graph_features(G)[None])[0]
    return TAU_CLASSES[pred[3]], PUSH_CLASSES[pred[4]]


def per_block_lb(model, P):
    """The load-balancing variant of every subgraph of an unstaged partition, from the
    subgraph's own features (the LB head), as tc_part_set_lb's warp thresholds."""
    lb_c = model.predict(part_features(P))[:, 1]
    wmin = [LB_WARP_MIN[LB_CLASSES[c]] for c in lb_c]
    P.set_lb(wmin)
    return wmin


def time_choice(G, choice, iters=5, reps=3):
    direction, block, lb = choice
    if block == "l2":
        P = tocab_partition(G, L.TC_PULL if direction == "pull" else L.TC_PUSH, 0)
        return time_config(G, direction, None, lb, iters, reps, part=P)
    return time_config(G, direction, block, lb, iters, reps)


# ------------------------------------------------------------------------------------------------
# training data: seeded synthetic graphs of four families, timed on the device
# ------------------------------------------------------------------------------------------------

def graph_specs(count: int, seed: int = 1000, scale_lo: int = 14, scale_hi: int = 20):
    """`count` seeded graph descriptions: R-MAT (varied skew), Erdos-Renyi, power-law
    configuration model (exponent 2.1-2.9) and 2D grids, scales in [scale_lo, scale_hi]."""
    import graphgen as gg
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        kind = ["rmat", "er", "plc", "grid"][i % 4]
        s = int(rng.integers(scale_lo, scale_hi + 1))
        ef = int(rng.choice([4, 8, 16, 32]))
        if kind == "rmat":
            a = float(rng.uniform(0.45, 0.65))
            b = c = (1.0 - a) / 3.0 * float(rng.uniform(0.8, 1.1))
            specs.append({"kind": "rmat", "scale": s, "ef": ef, "a": a, "b": b, "c": c, "seed": seed + i,
                          "permute": bool(rng.integers(0, 4) > 0)})
        elif kind == "er":
            specs.append({"kind": "er", "V": 1 << s, "M": ef << s, "seed": seed + i})
        elif kind == "plc":
            specs.append({"kind": "plc", "V": 1 << s, "avg": float(ef), "exp": float(rng.uniform(2.1, 2.9)),
                          "seed": seed + i})
        else:
            side = int(2 ** (s / 2))
            specs.append({"kind": "grid", "rows": side, "cols": side, "drop": float(rng.uniform(0, 0.2)),
                          "seed": seed + i})
    del gg
    return specs


def make_graph(spec, device="cuda"):
    import graphgen as gg
    k = spec["kind"]
    if k == "rmat":
        return gg.rmat(spec["scale"], spec["ef"], spec["a"], spec["b"], spec["c"], seed=spec["seed"],
                       permute_seed=7 if spec.get("permute", True) else None, device=device)
    if k == "er":
        return gg.erdos_renyi(spec["V"], spec["M"], seed=spec["seed"], device=device)
    if k == "plc":
        return gg.powerlaw_config(spec["V"], spec["avg"], spec["exp"], seed=spec["seed"], device=device)
    return gg.grid2d(spec["rows"], spec["cols"], drop=spec["drop"], seed=spec["seed"], device=device)


def _bfs_sources(g, n: int = 2):
    import graphgen as gg
    return [int(x) for x in gg.sources(g, n, seed=g.V)]


def build_dataset(specs, iters=5, reps=3, log=None):
    X, Y, tables = [], [], []
    for i, spec in enumerate(specs):
        g = make_graph(spec)
        G = graph_load_csr(g.rowptr, g.colidx, V=g.V)
        f = graph_features(G)
        m = measure_graph(G, iters=iters, reps=reps, bfs_src=_bfs_sources(g))
        X.append(f)
        Y.append(m["labels"])
        tables.append(m["table"])
        if log:
            log(f"[{i + 1}/{len(specs)}] {spec['kind']} V={g.V} E={g.E} labels={m['labels']}")
        del G, g
        torch.cuda.empty_cache()
    return np.asarray(X, np.float32), np.asarray(Y, np.int32), tables


def evaluate(model, specs, iters=5, reps=3, log=None):
    """Per graph: time of the model's choice, of the heuristic and of the exhaustive best."""
    rows = []
    for spec in specs:
        g = make_graph(spec)
        G = graph_load_csr(g.rowptr, g.colidx, V=g.V)
        m = measure_graph(G, iters=iters, reps=reps, bfs_src=_bfs_sources(g))
        pr = {k: v for k, v in m["table"].items() if not k.startswith("bfs|")}
        bt = {k: v for k, v in m["table"].items() if k.startswith("bfs|")}
        best = min(pr.values())
        heur = pr["pull|l2|hybrid"]
        ch = choose(model, G) if model is not None else heuristic_config()
        key = f"{ch[0]}|{ch[1]}|{ch[2]}"
        t_model = pr.get(key)
        if t_model is None:
            t_model = time_choice(G, ch, iters, reps)
        tau, push = choose_bfs(model, G) if model is not None else BFS_HEURISTIC
        bkey = f"bfs|{tau:g}|{push:.4g}"
        hkey = f"bfs|{BFS_HEURISTIC[0]:g}|{BFS_HEURISTIC[1]:.4g}"
        rows.append({"spec": spec, "V": g.V, "E": g.E, "choice": key, "t_model": t_model, "t_heuristic": heur,
                     "t_best": best, "bfs_choice": bkey, "bfs_model": bt.get(bkey), "bfs_heuristic": bt[hkey],
                     "bfs_best": min(bt.values())})
        if log:
            log(f"{spec['kind']} V={g.V} E={g.E}: model {key} {t_model:.4f} ms, heuristic {heur:.4f}, best {best:.4f}; "
                f"BFS {bkey} {bt.get(bkey)} heuristic {bt[hkey]:.4f} best {min(bt.values()):.4f}")
        del G, g
        torch.cuda.empty_cache()
    return rows


def _main():
    import argparse
    import sys
    import time
    ap = argparse.ArgumentParser(description="train the cost model on timings of generated graphs")
    ap.add_argument("--graphs", type=int, default=320)
    ap.add_argument("--scale-lo", type=int, default=14)
    ap.add_argument("--scale-hi", type=int, default=20)
    ap.add_argument("--heldout", type=int, default=24)
    ap.add_argument("--large", type=int, default=0, help="extra training graphs at scales 21-24")
    ap.add_argument("--large-heldout", type=int, default=0)
    ap.add_argument("--rmat25", action="store_true", help="add R-MAT scale 25 to the held-out set")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None)
    a = ap.parse_args()
    t0 = time.time()
    log = lambda s: print(s, file=sys.stderr, flush=True)  # noqa: E731
    specs = graph_specs(a.graphs, 1000, a.scale_lo, a.scale_hi) + graph_specs(a.large, 2000, 21, 24)
    X, Y, tables = build_dataset(specs, log=log)
    m = MLP()
    m.init(seed=0)
    loss = m.train(X, Y, epochs=a.epochs, batch=64, lr=3e-3)
    acc = (m.predict(X) == Y).mean(axis=0).tolist()
    hspecs = graph_specs(a.heldout, 900000, a.scale_lo, a.scale_hi) + graph_specs(a.large_heldout, 910000, 21, 24)
    if a.rmat25:
        hspecs.append({"kind": "rmat", "scale": 25, "ef": 16, "a": 0.57, "b": 0.19, "c": 0.19, "seed": 25,
                       "permute": True})
    held = evaluate(m, hspecs, log=log)
    gm = lambda k: float(np.exp(np.mean([np.log(r[k] / r["t_best"]) for r in held])))  # noqa: E731
    gmb = lambda k: float(np.exp(np.mean([np.log(r[k] / r["bfs_best"]) for r in held  # noqa: E731
                                          if r[k] is not None])))
    meta = {"graphs": a.graphs, "scales": [a.scale_lo, a.scale_hi], "large_graphs": a.large,
            "final_loss": loss, "train_accuracy": acc,
            "heldout": a.heldout, "heldout_model_over_best": gm("t_model"),
            "heldout_heuristic_over_best": gm("t_heuristic"),
            "heldout_bfs_model_over_best": gmb("bfs_model"), "heldout_bfs_heuristic_over_best": gmb("bfs_heuristic"),
            "seconds": time.time() - t0}
    m.save(a.out, meta)
    log(json.dumps(meta))
    if a.report:
        with open(a.report, "w") as fh:
            json.dump({"meta": meta, "heldout": held, "train_X": X.tolist(), "train_Y": Y.tolist(),
                       "tables": tables}, fh)


if __name__ == "__main__":
    _main()
