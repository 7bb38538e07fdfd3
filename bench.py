"""Benchmark of the TOCAB hot path on GB300.

Headline (one JSON line on rank 0): pull PageRank with TOCAB, 20 iterations, damping 0.85,
on a seeded R-MAT graph of scale 24 (edge factor 16, a=.57 b=.19 c=.19, relabelled,
self loops and duplicates removed).  metric = GTEPS = 20 * E / (time of one 20-iteration
run).  A "step" is one such run with the graph already resident in HBM.  The column
indices (about 1 GB) are larger than the 135 MB L2, so every step streams from HBM.

Also reported: unblocked pull, TOCAB/unblocked push and pull BFS (64 sources, symmetrised
R-MAT 24) as variants, the roofline of the dominant kernel (the pull gather), the e2e
number through the C ABI with host buffers, the FP64 oracle on the host cores
(cpu_baseline), and SM clocks sampled during the timed region.

--impl reference times the FP64 CPU oracle (the only reference implementation of the
method) on the same graph, on a bounded sample of iterations.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

ITERS = 20
DAMPING = 0.85
METRIC = "PageRank/BFS GTEPS on 1 GB300, TOCAB vs unblocked; % of HBM-bound roofline"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tocab", choices=["tocab", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--blocks", type=int, default=0, help="TOCAB block count (0 = from --policy)")
    ap.add_argument("--policy", default="smem", choices=["smem", "l2"],
                    help="block width when --blocks 0: one CTA's shared memory, or the paper's L2 rule")
    ap.add_argument("--bfs-sources", type=int, default=64)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--merge", default="fixed", choices=["fixed", "ordered"],
                    help="TOCAB pull merge: fixed-point or ordered (both deterministic)")
    ap.add_argument("--merge-range", type=int, default=0, help="vertices per merge CTA (0 = library default)")
    ap.add_argument("--order", default="outdegree", choices=["outdegree", "natural"],
                    help="vertex numbering the TOCAB blocks are cut in (renumbered by out-degree, or as given)")
    ap.add_argument("--quick", action="store_true",
                    help="headline only: skip variants, e2e and the CPU baseline (profiling runs)")
    ap.add_argument("--row", default="", choices=["", "many_graphs", "spmv", "bc", "bfs_grid", "rmat16", "ppr",
                                                  "ppr_probe", "ppr_probe_tile32", "bfs_levels"],
                    help="profiling runs: time only this row and print its figures")
    return ap.parse_args()


# --------------------------------------------------------------------------------------------
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch, from one single-pass ncu
# capture of `bench.py --steps 2 --warmup 1 --quick` on the full workload.  Keyed by kernel, R-MAT
# scale and block count, and tied to the sources it was taken on (SHA-256 over the files that
# define the two kernels, the partition and staged format they read, the graph preprocessing
# before it and the device helpers they use): after any change to those the figure no longer
# describes the kernels and the bench reports null.
NCU_TRAFFIC = {("k_tile_gather", 24, 179): 784667392,  # mean of two launches (786.0 and 783.3 MB)
               ("k_pull_merge_atomic<2>", 24, 179): 349975296}  # (349.8 and 350.1 MB)
NCU_TRAFFIC_SRC = "b4977289e92a6a36"


PULL_PATH_SOURCES = ("tc_common_dev.cuh", "tc_graph.cu", "tc_pagerank.cu", "tc_partition.cu", "tc_prims.cu",
                     "tc_tile.cu")


def library_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1904_02241_gb300", "csrc")
    for name in PULL_PATH_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, scale: int, blocks: int):
    if NCU_TRAFFIC_SRC != library_source_hash():
        return None
    return NCU_TRAFFIC.get((kernel, scale, blocks))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------------------------
def make_graph(scale: int, device: str):
    return gg.rmat(scale, device=device)


def time_runs(fn, steps: int, stream) -> list[float]:
    """Per-step device times (ms) of fn() with CUDA events on `stream`."""
    out = []
    for _ in range(steps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        out.append(s.elapsed_time(e))
    return out


def bench_tocab(args, world, rank, local):
    import paper_1904_02241_gb300 as T
    T.lib()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    g = make_graph(args.scale, "cuda")
    V, E = g.V, g.E
    gen_s = time.time() - t0
    G = T.graph_load_csr(g.rowptr, g.colidx, V=V)
    P = T.tocab_partition(G, T.TC_PULL, args.blocks, block_policy=args.policy, merge_range=args.merge_range,
                          order=args.order)
    torch.cuda.synchronize()
    out = torch.empty(V, dtype=torch.float32, device=dev)

    def step():
        T.pagerank_pull(G, P, damping=DAMPING, iters=ITERS, out=out, merge=args.merge)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        step()
    end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms_total = start.elapsed_time(end)
    # per-kernel durations over an identical set of steps, timed by the library with events
    prof = [T.pagerank_pull(G, P, damping=DAMPING, iters=ITERS, out=out, profile=True, return_stats=True,
                            merge=args.merge)[1]
            for _ in range(max(3, min(args.steps, 5)))]
    clk = clocks.stop()
    ms_step = max_over_ranks(ms_total / args.steps, world)
    edges_all = sum_over_ranks(float(E) * ITERS, world)
    value = edges_all / (ms_step * 1e-3) / 1e9

    gather_ms = statistics.median(p.ms_gather for p in prof) / ITERS
    merge_ms = statistics.median(p.ms_merge for p in prof) / ITERS
    launches_per_step = prof[0].launches

    # algorithmic bytes of one gather launch (Alg. 4 over all blocks), for the format in use:
    #   staged : 2 B per (padded) edge of block-relative sources + 1 bit row-start mask,
    #            each contribution read once (4V), partial sums written (4R)
    #   unstaged: 4 B per edge (global sources), 4(R+1) row offsets, 4V, 4R
    R = P.num_rows
    if P.staged:
        gather_bytes = 2 * P.staged_edges + P.staged_edges // 8 + 4 * V + 4 * R
        kname = "k_tile_gather"
    else:
        gather_bytes = 4 * E + 4 * (R + 1) + 4 * V + 4 * R
        kname = "k_pull_gather<false>"
    # merge: partial sums (4 B) and local ids (2 B) per local row, the range table, and the out-degree
    # reciprocal read and contribution written per vertex with out-edges (renumbered: the others
    # are skipped; natural order: every vertex)
    per_vertex = 8 * (P.num_sources if P.vertex_order == T.TC_ORDER_OUTDEGREE else V)
    merge_bytes = 6 * R + 8 * P.num_blocks * (P.num_ranges + 1) + per_vertex
    peak, peak_kind = load_peaks()
    # Roofline of the dominant kernel (the gather), against the method-independent bytes that
    # its part of an iteration must move: every column index (4E) and every contribution (4V).
    # The kernel's own format moves 2 B per staged edge instead, plus row heads and partial sums:
    # reported beside as own_format_*.  The whole iteration against B_min is the headline figure.
    gather_bmin = 4 * E + 4 * V
    achieved = gather_bmin / (gather_ms * 1e-3) / 1e9
    bmin = 4 * E + 4 * (V + 1) + 4 * V + 4 * V + 4 * V
    res = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": "GTEPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"pagerank_pull_tocab rmat{args.scale} ef16 20 iters d=0.85",
                   "merge": args.merge, "merge_range": P.merge_range, "vertex_order": args.order,
                   "graph": f"rmat{args.scale}", "V": V, "E": E, "iters": ITERS,
                   "blocks": P.num_blocks, "block_width": P.block_width, "local_rows": R,
                   "l2": "inputs larger than L2 (colidx %.2f GB vs 135 MB L2); no flush" % (4 * E / 1e9),
                   "parallelism": f"replicas x{world}", "generate_s": round(gen_s, 2)},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1),
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": ncu_traffic(kname, args.scale, P.num_blocks),
                     "algorithmic_bytes": gather_bmin,
                     "headline": "iteration_bmin_frac",
                     "iteration_bmin_frac": round(bmin / (ms_step / ITERS * 1e-3) / 1e9 / peak, 4),
                     "iteration_bmin_bytes": bmin,
                     "own_format_bytes": gather_bytes,
                     "own_format_frac": round(gather_bytes / (gather_ms * 1e-3) / 1e9 / peak, 4),
                     "gather_ms": round(gather_ms, 4), "merge_ms": round(merge_ms, 4),
                     "merge_traffic": ncu_traffic("k_pull_merge_atomic<2>", args.scale, P.num_blocks),
                     "merge_gbs": round(merge_bytes / (merge_ms * 1e-3) / 1e9, 1)},
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
    }
    del prof
    return res, (g, G, P, out, stream)


def variants(args, ctx, world):
    """Unblocked pull, push (unblocked and TOCAB), pull BFS: GTEPS of each."""
    import paper_1904_02241_gb300 as T
    g, G, P, out, stream = ctx
    E = g.E
    steps = max(3, min(args.steps, 5))
    res = {}

    def run(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        return statistics.median(time_runs(fn, steps, stream))

    peak, _ = load_peaks()
    V = g.V
    bmin = 4 * E + 4 * (V + 1) + 12 * V  # method-independent bytes of one iteration

    def bmin_frac(ms_run):
        return round(bmin / (ms_run / ITERS * 1e-3) / 1e9 / peak, 4)

    ms = run(lambda: T.pagerank_pull(G, None, damping=DAMPING, iters=ITERS, out=out))
    res["pull_unblocked_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res["pull_unblocked_bmin_frac"] = bmin_frac(ms)
    res["pull_tocab_blocks"] = P.num_blocks
    other_order = "natural" if args.order == "outdegree" else "outdegree"
    Pn = T.tocab_partition(G, T.TC_PULL, args.blocks, block_policy=args.policy, order=other_order)
    ms = run(lambda: T.pagerank_pull(G, Pn, damping=DAMPING, iters=ITERS, out=out))
    res[f"pull_tocab_{other_order}_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res[f"pull_tocab_{other_order}_bmin_frac"] = bmin_frac(ms)
    res[f"pull_tocab_{other_order}_local_rows"] = Pn.num_rows
    del Pn
    other = "l2" if args.policy == "smem" else "smem"
    Po = T.tocab_partition(G, T.TC_PULL, 0, block_policy=other)
    ms = run(lambda: T.pagerank_pull(G, Po, damping=DAMPING, iters=ITERS, out=out))
    res[f"pull_tocab_{other}_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res[f"pull_tocab_{other}_bmin_frac"] = bmin_frac(ms)
    res[f"pull_tocab_{other}_blocks"] = Po.num_blocks
    # the unstaged gathers again, with an L2 access-policy window over the contributions
    ms = run(lambda: T.pagerank_pull(G, None, damping=DAMPING, iters=ITERS, out=out, l2_window=True))
    res["pull_unblocked_l2window_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    if other == "l2":
        ms = run(lambda: T.pagerank_pull(G, Po, damping=DAMPING, iters=ITERS, out=out, l2_window=True))
        res["pull_tocab_l2_l2window_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    del Po
    Pp = T.tocab_partition(G, T.TC_PUSH, args.blocks, block_policy="l2")
    ms = run(lambda: T.pagerank_push(G, Pp, damping=DAMPING, iters=ITERS, out=out))
    res["push_tocab_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res["push_tocab_bmin_frac"] = bmin_frac(ms)
    ms = run(lambda: T.pagerank_push(G, None, damping=DAMPING, iters=ITERS, out=out))
    res["push_unblocked_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res["push_unblocked_bmin_frac"] = bmin_frac(ms)
    # the paper's FP32 atomics instead of the default 64-bit fixed-point reductions, and the
    # thread/warp/CTA row mapping instead of the edge-parallel scatter
    push = {}
    for key, P_, kw in (("tocab_float", Pp, {"sums": "float"}), ("unblocked_float", None, {"sums": "float"}),
                        ("unblocked_twc_fixed", None, {"lb_warp_min": 32}),
                        ("unblocked_twc_float", None, {"lb_warp_min": 32, "sums": "float"})):
        ms = run(lambda: T.pagerank_push(G, P_, damping=DAMPING, iters=ITERS, out=out, **kw))
        push[key + "_gteps"] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
    res["push_variants"] = push
    del Pp
    # direct pieces (single-edge pieces of the first blocks added by the merge): an opt-in
    # partition option, measured against the default here
    if args.order == "outdegree":
        Pd = T.tocab_partition(G, T.TC_PULL, args.blocks, block_policy=args.policy, merge_range=args.merge_range,
                               order="outdegree", direct_blocks=-1)
        ms = run(lambda: T.pagerank_pull(G, Pd, damping=DAMPING, iters=ITERS, out=out))
        res["pull_tocab_direct_pieces"] = {"gteps": round(E * ITERS / (ms * 1e-3) / 1e9, 2),
                                           "bmin_frac": bmin_frac(ms), "direct_blocks": Pd.direct_blocks,
                                           "num_direct": Pd.num_direct, "local_rows": Pd.num_rows}
        del Pd
    # BFS on the symmetrised graph, 64 seeded sources (TEPS counts each undirected edge once)
    gs = gg.symmetrize(g)
    Gs = T.graph_load_csr(gs.rowptr, gs.colidx, V=gs.V)
    Ps = T.tocab_partition(Gs, T.TC_PULL, args.blocks, block_policy="l2")
    lv = torch.empty(gs.V, dtype=torch.int32, device="cuda")
    srcs = gg.sources(gs, args.bfs_sources, seed=13)
    # pure pull (the paper's topology-driven BFS): TOCAB with 8 blocks, every level blocked (the
    # best of the block and threshold sweeps below), against unblocked; then the same with the
    # L2-rule blocks and tau = 0.05, and direction-optimised levels
    P8 = T.tocab_partition(Gs, T.TC_PULL, 8, smem_stage=-1)
    res["bfs_tocab_gteps"] = bfs_rate(T, Gs, P8, srcs, lv, stream, 0.0, 0.0)[0]
    res["bfs_tocab_config"] = {"blocks": P8.num_blocks, "tocab_threshold": 0.0}
    del P8
    for thr, push, key in [(-1.0, 0.0, "bfs_unblocked"), (0.05, 0.0, "bfs_tocab_l2_tau0.05"),
                           (0.05, 1.0 / 24, "bfs_diropt_tocab"), (-1.0, 1.0 / 24, "bfs_diropt_unblocked")]:
        res[key + "_gteps"] = bfs_rate(T, Gs, Ps, srcs, lv, stream, thr, push)[0]
    # the small-frontier push levels host-driven, one launch sequence and round trip per level
    res["bfs_diropt_unblocked_no_resident_gteps"] = bfs_rate(T, Gs, Ps, srcs, lv, stream, -1.0, 1.0 / 24, 0)[0]
    res["bfs_graph"] = {"V": gs.V, "E_directed": gs.E, "sources": len(srcs)}
    res["bfs_oracle"] = oracle_bfs_rate(gs, srcs[0])
    # the TOCAB frontier threshold tau (Sec. 3.3, "frontier large enough"), swept on 16 of the
    # sources: pure pull levels and direction-optimised levels; levels are identical for every tau
    res["bfs_tau_sweep_gteps"] = bfs_tau_sweep(T, Gs, Ps, srcs[:16], lv, stream)
    taus = res["bfs_tau_sweep_gteps"]
    res["bfs_tau_best"] = {kind: max(taus[kind], key=lambda k: taus[kind][k]) for kind in taus}
    # pure pull BFS (the paper's topology-driven form) with every level blocked, over block
    # counts: blocks whose frontier-bitmap slice stays in L1 turn the full-scan levels' random
    # bitmap reads into L1 hits
    bsweep = {}
    for B in (8, 32, 128):
        Pb = T.tocab_partition(Gs, T.TC_PULL, B, smem_stage=-1)
        bsweep[str(B)] = bfs_rate(T, Gs, Pb, srcs[:16], lv, stream, 0.0, 0.0)[0]
        del Pb
    res["bfs_pull_blocked_by_blocks_gteps"] = bsweep
    del Gs, Ps, gs, lv
    torch.cuda.empty_cache()
    # block-count sweep around the L2 capacity (paper's source-range blocks, unstaged gather)
    sweep = {}
    for B in (1, 2, 4, 8, 16, 32, 64):
        Pb = T.tocab_partition(G, T.TC_PULL, B)
        ms = run(lambda: T.pagerank_pull(G, Pb, damping=DAMPING, iters=ITERS, out=out))
        sweep[str(B)] = round(E * ITERS / (ms * 1e-3) / 1e9, 2)
        del Pb
    res["pull_tocab_block_sweep_gteps"] = sweep
    torch.cuda.empty_cache()
    res["rmat16"] = rmat16_row(stream, run)
    res["bfs_grid4096"] = bfs_grid_row(stream)
    res.update(spmv_row(stream))
    res.update(bc_rows(stream))
    res.update(graph_variants(args, stream, E, run))
    res.update(batch_variants(args, stream))
    return res


def bfs_rate(T, G, P, srcs, lv, stream, thr, push, resident=-1):
    """GTEPS of BFS from every source (edges reached / 2, symmetrised graphs) and the levels."""
    T.bfs_pull(G, P, srcs[0], tocab_threshold=thr, out=lv, push_threshold=push, resident_edges=resident)
    torch.cuda.synchronize()
    tot_ms, tot_edges, levels = 0.0, 0, 0
    for s in srcs:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        _, st = T.bfs_pull(G, P, s, tocab_threshold=thr, out=lv, return_stats=True, push_threshold=push,
                           resident_edges=resident)
        t1.record(stream)
        t1.synchronize()
        tot_ms += t0.elapsed_time(t1)
        tot_edges += st.edges_reached // 2
        levels = max(levels, st.levels)
    return round(tot_edges / (tot_ms * 1e-3) / 1e9, 2), levels


def bfs_tau_sweep(T, G, P, srcs, lv, stream):
    out = {}
    for kind, push in (("pull", 0.0), ("diropt", 1.0 / 24)):
        out[kind] = {}
        for tau in (0.0, 0.02, 0.05, 0.1, 0.2, 0.4, -1.0):
            out[kind][str(tau)] = bfs_rate(T, G, P, srcs, lv, stream, tau, push)[0]
    return out


def rmat16_row(stream, run):
    """The small configuration: R-MAT 16 (V = 65,536, ~1M edges), unblocked pull against TOCAB with
    4 source-range blocks (the paper's ranges, and the same after renumbering by out-degree)."""
    import paper_1904_02241_gb300 as T
    g = gg.rmat(16, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    out = torch.empty(g.V, dtype=torch.float32, device="cuda")
    row = {"V": g.V, "E": g.E}
    for key, P in (("pull_unblocked", None), ("pull_tocab_b4", T.tocab_partition(G, T.TC_PULL, 4)),
                   ("pull_tocab_b4_renumbered", T.tocab_partition(G, T.TC_PULL, 4, order="outdegree"))):
        ms = run(lambda: T.pagerank_pull(G, P, damping=DAMPING, iters=ITERS, out=out))
        row[key + "_gteps"] = round(g.E * ITERS / (ms * 1e-3) / 1e9, 2)
    return row


def bfs_grid_row(stream, nsrc: int = 64):
    """BFS on the 4096 x 4096 grid with 5% of its edges removed (both directions): about 8,000
    levels with small frontiers, so the levels run top-down (direction optimisation), by default
    inside cluster-resident launches; pure pull levels rescan every unvisited vertex per level
    and are not timed here."""
    import paper_1904_02241_gb300 as T
    g = gg.grid2d(4096, 4096, drop=0.05, seed=11, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="l2")
    lv = torch.empty(g.V, dtype=torch.int32, device="cuda")
    srcs = gg.sources(g, nsrc, seed=13)
    row = {"V": g.V, "E_directed": g.E, "sources": nsrc}
    for key, thr, res in (("bfs_diropt_unblocked", -1.0, -1), ("bfs_diropt_tocab", 0.05, -1),
                          ("bfs_diropt_unblocked_no_resident", -1.0, 0)):
        gteps, levels = bfs_rate(T, G, P, srcs if res else srcs[:2], lv, stream, thr, 1.0 / 24, res)
        row[key + "_gteps"] = gteps
        row["levels_max"] = levels
    row["no_resident_sources"] = 2
    return row


def graph_variants(args, stream, E_rmat, run):
    """The other two graph shapes of the PageRank workload: an Erdos-Renyi graph with the R-MAT's
    vertex and edge count, and the 4096 x 4096 grid with 5% of its edges removed.  Pull TOCAB
    (the default block policy, in the graph's own numbering and renumbered), unblocked pull, push
    TOCAB and unblocked on each, and the pull block-count sweep 1-64."""
    import paper_1904_02241_gb300 as T
    peak, _ = load_peaks()
    res = {}
    V24 = 1 << args.scale
    for name, make in (("er", lambda: gg.erdos_renyi(V24, E_rmat, seed=3, device="cuda")),
                       ("grid4096", lambda: gg.grid2d(4096, 4096, drop=0.05, seed=11, device="cuda"))):
        g = make()
        G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
        P = T.tocab_partition(G, T.TC_PULL, args.blocks, block_policy=args.policy)
        Pr = T.tocab_partition(G, T.TC_PULL, args.blocks, block_policy=args.policy, order="outdegree")
        out = torch.empty(g.V, dtype=torch.float32, device="cuda")
        bmin = 4 * g.E + 4 * (g.V + 1) + 12 * g.V
        row = {"V": g.V, "E": g.E, "blocks": P.num_blocks}
        Pp = T.tocab_partition(G, T.TC_PUSH, 0)
        for key, fn in (("pull_tocab", lambda: T.pagerank_pull(G, P, damping=DAMPING, iters=ITERS, out=out)),
                        ("pull_tocab_renumbered", lambda: T.pagerank_pull(G, Pr, damping=DAMPING, iters=ITERS,
                                                                          out=out)),
                        ("pull_unblocked", lambda: T.pagerank_pull(G, None, damping=DAMPING, iters=ITERS, out=out)),
                        ("push_tocab", lambda: T.pagerank_push(G, Pp, damping=DAMPING, iters=ITERS, out=out)),
                        ("push_unblocked", lambda: T.pagerank_push(G, None, damping=DAMPING, iters=ITERS, out=out))):
            ms = run(fn)
            row[key + "_gteps"] = round(g.E * ITERS / (ms * 1e-3) / 1e9, 2)
            row[key + "_bmin_frac"] = round(bmin / (ms / ITERS * 1e-3) / 1e9 / peak, 4)
        row["push_tocab_blocks"] = Pp.num_blocks
        del Pp, P, Pr
        # the paper's source-range blocks (unstaged gather) over block counts 1-64
        sweep = {}
        for B in (1, 2, 4, 8, 16, 32, 64):
            Pb = T.tocab_partition(G, T.TC_PULL, B)
            ms = run(lambda: T.pagerank_pull(G, Pb, damping=DAMPING, iters=ITERS, out=out))
            sweep[str(B)] = round(g.E * ITERS / (ms * 1e-3) / 1e9, 2)
            del Pb
        row["pull_tocab_block_sweep_gteps"] = sweep
        res[name] = row
        del G, g, out
        torch.cuda.empty_cache()
    return res


def batch_variants(args, stream):
    """Batching: 256 personalised PageRank sources on R-MAT 22 (all iterations in one persistent,
    graph-captured launch with the autotuned hot block and width), and 1,000 R-MAT graphs with
    scales 10..16 in one persistent, graph-captured launch with the lanes-per-vertex variant
    chosen by the autotuner."""
    res = ppr_row(stream)
    res.update(many_graphs(stream))
    return res


def ppr_row(stream):
    """256 personalised PageRank sources on R-MAT 22: the persistent batch (autotuned first) and
    the TOCAB-blocked form per 32-column tile."""
    import paper_1904_02241_gb300 as T
    res = {}
    g22 = gg.rmat(22, device="cuda")
    G22 = T.graph_load_csr(g22.rowptr, g22.colidx, V=g22.V)
    srcs = gg.sources(g22, 256, seed=17)
    R = torch.empty((g22.V, 256), dtype=torch.float32, device="cuda")
    hot, tile, tune_ms = T.ppr_autotune(G22, srcs)
    T.ppr_batch(G22, srcs, iters=ITERS, out=R)
    torch.cuda.synchronize()
    ms = statistics.median(time_runs(lambda: T.ppr_batch(G22, srcs, iters=ITERS, out=R), 3, stream))
    peak, _ = load_peaks()
    V22, E22, NP = g22.V, g22.E, 256
    # bytes of one iteration: without reuse every in-edge reads its source's 1 KB row; the
    # floor reads every row once (the whole [V x 256] matrix in, the next one out)
    row_bytes = 4 * E22 + 4 * (V22 + 1) + 4 * NP * E22 + 8 * V22 * NP
    floor_bytes = 4 * E22 + 4 * V22 + 2 * 4 * NP * V22
    res["ppr_oracle"] = oracle_ppr_rate(g22, srcs[0])
    res["ppr_batch"] = {"graph": "rmat22", "V": V22, "E": E22, "sources": 256, "iters": ITERS,
                        "ms": round(ms, 2), "ms_per_iter": round(ms / ITERS, 3),
                        "launches_per_run": 1, "cuda_graph": True,
                        "autotuned": {"hot_rows": hot, "tile_columns": tile,
                                      "ms_3_iters": {f"tile{w or 'whole'}_l2frac{f:g}": round(t, 3)
                                                     for (w, f), t in tune_ms.items()}},
                        "edge_columns_per_s_G": round(E22 * 256 * ITERS / (ms * 1e-3) / 1e9, 1),
                        "gteps_equiv": round(E22 * ITERS / (ms * 1e-3) / 1e9, 3),
                        "row_bytes_frac": round(row_bytes / (ms / ITERS * 1e-3) / 1e9 / peak, 4),
                        "floor_bytes_frac": round(floor_bytes / (ms / ITERS * 1e-3) / 1e9 / peak, 4)}
    # TOCAB per 32-column tile: source blocks whose 128-byte row segments fit in L2
    P22 = T.tocab_partition(G22, T.TC_PULL, 0, l2_fraction=1.0 / 88, merge_range=256)
    T.ppr_batch(G22, srcs, iters=ITERS, out=R, part=P22)
    torch.cuda.synchronize()
    ms = statistics.median(time_runs(lambda: T.ppr_batch(G22, srcs, iters=ITERS, out=R, part=P22), 3, stream))
    res["ppr_batch_tocab"] = {"blocks": P22.num_blocks, "block_width": P22.block_width, "ms": round(ms, 2),
                              "ms_per_iter": round(ms / ITERS, 3),
                              "edge_columns_per_s_G": round(g22.E * 256 * ITERS / (ms * 1e-3) / 1e9, 1),
                              "gteps_equiv": round(g22.E * ITERS / (ms * 1e-3) / 1e9, 3),
                              "floor_bytes_frac": round(floor_bytes / (ms / ITERS * 1e-3) / 1e9 / peak, 4)}
    del R, G22, g22, P22
    torch.cuda.empty_cache()
    return res


def many_graphs(stream, with_oracle: bool = True):
    """1,000 R-MAT graphs with scales 10..16, all iterations in one persistent, graph-captured
    launch with the variant chosen by the autotuner."""
    import paper_1904_02241_gb300 as T
    res = {}
    peak, _ = load_peaks()
    scales = gg.batch_scales(1000, 10, 16, seed=19)
    gb, off = gg.rmat_batch(scales, seed=19, device="cuda")
    M = T.multigraph_load(gb.rowptr, gb.colidx, off)
    best, times = T.multi_autotune(M, iters=ITERS)
    out = torch.empty(gb.V, dtype=torch.float32, device="cuda")
    T.pagerank_multi(M, iters=ITERS, out=out)
    torch.cuda.synchronize()
    ms = statistics.median(time_runs(lambda: T.pagerank_multi(M, iters=ITERS, out=out), 5, stream))
    if with_oracle:
        res["many_graphs_oracle"] = oracle_multi_rate(gb, off)
    # the resident kernel's bytes per iteration: 2 B of source and 1/8 B of head bits per
    # stream edge (the in-edges plus one placeholder per vertex without in-edges) and the
    # out-degree reciprocal of every vertex
    empties = int((torch.bincount(gb.colidx.long(), minlength=gb.V) == 0).sum())
    res_bytes = 2.125 * (gb.E + empties) + 4 * gb.V
    res["many_graphs"] = {"graphs": 1000, "scales": "U{10..16}", "V": gb.V, "E": gb.E, "iters": ITERS,
                          "autotuned_lanes_per_vertex": best, "autotune_ms": {str(k): round(v, 3) for k, v in times.items()},
                          "ms": round(ms, 3), "gteps": round(gb.E * ITERS / (ms * 1e-3) / 1e9, 2),
                          "bmin_frac": round((4 * gb.E + 4 * (gb.V + 1) + 12 * gb.V) / (ms / ITERS * 1e-3) / 1e9 / peak, 4),
                          "resident_bytes_frac": round(res_bytes / (ms / ITERS * 1e-3) / 1e9 / peak, 4)
                          if best == T.TC_MULTI_RESIDENT else None,
                          "launches_per_run": 1, "cuda_graph": True}
    del M, gb, out
    torch.cuda.empty_cache()
    return res


def ppr_probe_row(stream, tile: int = 0, iters: int = 3):
    """The PPR batch (256 sources, R-MAT 22) for a profiler: one warm call and one call of
    `iters` iterations with a fixed tile width (0: whole rows) and no evict-last rows."""
    import paper_1904_02241_gb300 as T
    g = gg.rmat(22, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    srcs = gg.sources(g, 256, seed=17)
    R = torch.empty((g.V, 256), dtype=torch.float32, device="cuda")
    T.ppr_set_tuning(G, hot=0, tile=tile)
    T.ppr_batch(G, srcs, iters=iters, out=R)
    _, st = T.ppr_batch(G, srcs, iters=iters, out=R, profile=True, return_stats=True)
    return {"ppr_probe": {"tile": tile, "iters": iters, "ms": round(st.ms_total, 3)}}


def bfs_levels_row(stream):
    """Pure pull BFS (no push levels) on the symmetrised R-MAT 22 from one source, unblocked
    (tocab_threshold -1) and with every level blocked (0): the per-level trace, for a profiler."""
    import paper_1904_02241_gb300 as T
    g = gg.symmetrize(gg.rmat(22, device="cuda"))
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    P = T.tocab_partition(G, T.TC_PULL, 8)
    src = gg.sources(g, 1, seed=13)[0]
    lv = torch.empty(g.V, dtype=torch.int32, device="cuda")
    out = {"V": g.V, "E": g.E, "blocks": P.num_blocks, "W": P.block_width}
    for tau in (-1.0, 0.0):
        _, st = T.bfs_pull(G, P, src, tocab_threshold=tau, out=lv, return_stats=True, profile=True)
        n = min(st.levels, 64)
        out[f"tau_{tau:g}"] = {"levels": st.levels, "ms": round(st.ms_total, 3),
                               "level_ms": [round(st.level_ms[i], 4) for i in range(n)],
                               "level_frontier": [int(st.level_frontier[i]) for i in range(n)]}
    return {"bfs_levels": out}


def spmv_row(stream, scale: int = 22):
    """y = A x with A the R-MAT 22 CSR and seeded FP32 values (Sec. 4's SpMV benchmark).  The
    algorithmic bytes of one product are the values and column indices (8 B per entry), the row
    offsets, x once and y: 8E + 4(V+1) + 8V."""
    import paper_1904_02241_gb300 as T
    g = gg.rmat(scale, device="cuda")
    A = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    vals = gg.edge_values(g).cuda()
    x = torch.randn(g.V, device="cuda")
    y = torch.empty(g.V, device="cuda")
    for _ in range(3):
        T.spmv(A, vals, x, out=y)
    torch.cuda.synchronize()
    ms = statistics.median(time_runs(lambda: T.spmv(A, vals, x, out=y), 10, stream))
    peak, _ = load_peaks()
    nbytes = 8 * g.E + 4 * (g.V + 1) + 8 * g.V
    # GC-pull (TOCAB with a value stream) over column blocks of several widths
    gc = {}
    for B in (1, 8, 32, 128):
        P = T.tocab_partition(A, T.TC_PUSH, B, merge_range=8192)
        T.part_set_values(P, vals)
        for _ in range(3):
            T.spmv_tocab(P, x, out=y)
        torch.cuda.synchronize()
        ms_b = statistics.median(time_runs(lambda: T.spmv_tocab(P, x, out=y), 10, stream))
        gc[str(B)] = {"ms": round(ms_b, 4), "local_rows": P.num_rows, "block_width": P.block_width}
        del P
    # GC-push (row blocks of y, FP32 atomic adds) over the same block counts
    gp = {}
    for B in (1, 8, 32, 128):
        P = T.tocab_partition(A, T.TC_PULL, B, smem_stage=-1)
        T.part_set_values(P, vals)
        for _ in range(3):
            T.spmv_tocab(P, x, out=y)
        torch.cuda.synchronize()
        ms_b = statistics.median(time_runs(lambda: T.spmv_tocab(P, x, out=y), 10, stream))
        gp[str(B)] = {"ms": round(ms_b, 4), "local_rows": P.num_rows, "block_width": P.block_width}
        del P
    return {"spmv": {"graph": f"rmat{scale}", "V": g.V, "E": g.E, "ms": round(ms, 4),
                     "gflops": round(2 * g.E / (ms * 1e-3) / 1e9, 2),
                     "bytes_frac": round(nbytes / (ms * 1e-3) / 1e9 / peak, 4),
                     "mapping": "lane groups per row (VWC) + CTA per hub row",
                     "gc_pull_by_blocks": gc, "gc_push_by_blocks": gp}}


def bc_rows(stream):
    """BC on the symmetrised R-MAT 18 (the earlier row) and 21 (vertex arrays beyond L1/L2 reach)."""
    return {"bc": bc_row(stream, 18)["bc"], "bc_rmat21": bc_row(stream, 21)["bc"]}


def bc_row(stream, scale: int = 18, nsrc: int = 4):
    """Betweenness centrality from a few seeded sources on the symmetrised R-MAT; TEPS counts each
    undirected edge once per source."""
    import paper_1904_02241_gb300 as T
    gs = gg.symmetrize(gg.rmat(scale, device="cuda"))
    G = T.graph_load_csr(gs.rowptr, gs.colidx, V=gs.V)
    srcs = gg.sources(gs, nsrc, seed=13)
    out = torch.empty(gs.V, dtype=torch.float64, device="cuda")
    T.bc(G, srcs[:1], out=out)
    torch.cuda.synchronize()
    ms = statistics.median(time_runs(lambda: T.bc(G, srcs, out=out), 3, stream))
    blocked = {}
    for B in (4, 16, 64):  # TOCAB pull levels (tc_bc_tocab): the same scores, bit for bit
        P = T.tocab_partition(G, T.TC_PULL, B, merge_range=8192, smem_stage=-1)
        T.bc(G, srcs[:1], out=out, part=P)
        torch.cuda.synchronize()
        ms_b = statistics.median(time_runs(lambda: T.bc(G, srcs, out=out, part=P), 3, stream))
        blocked[str(B)] = {"ms": round(ms_b, 3), "gteps": round(gs.E / 2 * nsrc / (ms_b * 1e-3) / 1e9, 3)}
        del P
    return {"bc": {"graph": f"rmat{scale}_sym", "V": gs.V, "E_directed": gs.E, "sources": nsrc, "ms": round(ms, 3),
                   "gteps": round(gs.E / 2 * nsrc / (ms * 1e-3) / 1e9, 3), "tocab_pull_levels_by_blocks": blocked}}


def e2e(args, ctx):
    """Same metric through the C ABI from host buffers: H2D of the CSR, graph load
    (validation + transpose), partition, 20 iterations, D2H of the ranks."""
    import paper_1904_02241_gb300 as T
    g, G, P, out, stream = ctx
    rp_h = g.rowptr.cpu().pin_memory()
    ci_h = g.colidx.cpu().pin_memory()
    out_h = torch.empty(g.V, dtype=torch.float32).pin_memory()

    def job():  # the headline's configuration, from host buffers to host ranks
        G2 = T.graph_load_csr(rp_h, ci_h, V=g.V)
        P2 = T.tocab_partition(G2, T.TC_PULL, args.blocks, block_policy=args.policy, merge_range=args.merge_range,
                               order=args.order)
        T.pagerank_pull(G2, P2, damping=DAMPING, iters=ITERS, out=out_h, merge=args.merge)
        del P2, G2

    for _ in range(max(args.warmup, 1)):  # untimed, like the headline's warm-up steps
        job()
    times = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        job()
        t1.record(stream)
        t1.synchronize()
        times.append(t0.elapsed_time(t1))
    ms = statistics.median(times)
    # the one-time preprocessing on its own (inputs already on the device)
    tl, tp = [], []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        P2 = T.tocab_partition(G2, T.TC_PULL, args.blocks, block_policy=args.policy, merge_range=args.merge_range,
                               order=args.order)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        tl.append((t1 - t0) * 1e3)
        tp.append((t2 - t1) * 1e3)
        del P2, G2
    return {"value": round(g.E * ITERS / (ms * 1e-3) / 1e9, 3), "unit": "GTEPS",
            "load_transpose_ms": round(statistics.median(tl), 2), "partition_ms": round(statistics.median(tp), 2),
            "h2d_bytes_per_step": int(rp_h.numel() * 4 + ci_h.numel() * 4),
            "d2h_bytes_per_step": int(out_h.numel() * 4), "ms_per_step": round(ms, 3),
            "includes": "H2D CSR + load/transpose + renumbering and partition + 20 iters + D2H ranks",
            "warmup": max(args.warmup, 1)}


# ---- the FP64 oracle timed beside the variant rows (bounded samples, single thread) ----------

def oracle_bfs_rate(gs, source):
    """The oracle's level-synchronous BFS from one source on the same symmetrised graph."""
    import oracle
    oracle.build()
    rp, ci = gs.numpy()
    t0 = time.time()
    lv = oracle.bfs(gs.V, rp, ci, source)
    dt = time.time() - t0
    edges = int(np.diff(rp)[lv >= 0].sum()) // 2
    return {"gteps": round(edges / dt / 1e9, 4), "cores": 1, "sample": "1 source (of the 64)"}


def oracle_ppr_rate(g, source):
    """The oracle's personalised PageRank for one column (of the 256) and 20 iterations."""
    import oracle
    oracle.build()
    rp, ci = g.numpy()
    tr = oracle.transpose(g.V, rp, ci)
    t0 = time.time()
    oracle.ppr_pull(g.V, rp, ci, [source], iters=ITERS, transposed=tr)
    dt = time.time() - t0
    return {"edge_columns_per_s_G": round(g.E * ITERS / dt / 1e9, 4), "cores": 1,
            "sample": "1 column (of the 256), 20 iterations"}


def oracle_multi_rate(gb, off, count: int = 50):
    """The oracle's PageRank on a seeded sample of the batch's graphs, one after the other."""
    import oracle
    oracle.build()
    rp, ci = gb.numpy()
    o = off.cpu().numpy().astype(np.int64)
    pick = np.random.default_rng(29).choice(len(o) - 1, size=min(count, len(o) - 1), replace=False)
    edges, t0 = 0, time.time()
    for k in pick:
        lo, hi = int(o[k]), int(o[k + 1])
        oracle.pagerank_pull(hi - lo, rp[lo:hi + 1] - rp[lo], ci[rp[lo]:rp[hi]] - lo, iters=ITERS)
        edges += int(rp[hi] - rp[lo])
    dt = time.time() - t0
    return {"gteps": round(edges * ITERS / dt / 1e9, 4), "cores": 1,
            "sample": f"{len(pick)} of the {len(o) - 1} graphs, 20 iterations each"}


def cpu_baseline(g, budget_s: float):
    """The FP64 oracle (Alg. 1) on the host cores, on a bounded number of iterations."""
    import oracle
    oracle.build()
    rp, ci = g.rowptr.cpu().numpy(), g.colidx.cpu().numpy()
    tr = oracle.transpose(g.V, rp, ci)
    cores = os.cpu_count() or 1
    t0 = time.time()
    oracle.pagerank_pull(g.V, rp, ci, iters=1, nthreads=cores, transposed=tr)
    one = time.time() - t0
    iters = max(1, min(ITERS, int(budget_s / max(one, 1e-3))))
    t0 = time.time()
    oracle.pagerank_pull(g.V, rp, ci, iters=iters, nthreads=cores, transposed=tr)
    dt = time.time() - t0
    return {"value": round(g.E * iters / dt / 1e9, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "sample": f"{iters} of the 20 FP64 pull iterations on the same rmat graph "
                      f"(V={g.V}, E={g.E}), OpenMP over destinations"}


def reference_arm(args, world, rank):
    if rank != 0:
        return
    t0 = time.time()
    g = gg.rmat_host(args.scale)  # the same graph as the GPU arm's, generated on the host cores
    gen_s = time.time() - t0
    import oracle
    oracle.build()
    rp, ci = g.rowptr.numpy(), g.colidx.numpy()
    tr = oracle.transpose(g.V, rp, ci)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.pagerank_pull(g.V, rp, ci, iters=1, nthreads=cores, transposed=tr)
    times = []
    for _ in range(args.steps):
        t0 = time.time()
        oracle.pagerank_pull(g.V, rp, ci, iters=1, nthreads=cores, transposed=tr)
        times.append(time.time() - t0)
    sec_iter = statistics.median(times)
    value = g.E / sec_iter / 1e9
    sample = f"1 FP64 pull iteration per step (of the 20) on rmat{args.scale} (V={g.V}, E={g.E})"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GTEPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec_iter * 1e3, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"pagerank_pull rmat{args.scale} ef16 20 iters d=0.85 (FP64 CPU oracle)",
                   "graph": f"rmat{args.scale}", "V": g.V, "E": g.E, "iters": ITERS,
                   "generated_on": "host (graphgen.rmat_host)", "generate_s": round(gen_s, 2)},
        "cpu_baseline": {"value": round(value, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the TOCAB path has no CPU fallback)")
    if args.row:
        stream = torch.cuda.current_stream()
        def run(fn):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            return statistics.median(time_runs(fn, 5, stream))
        res = {"many_graphs": lambda: many_graphs(stream, with_oracle=False), "spmv": lambda: spmv_row(stream),
               "bc": lambda: bc_rows(stream), "bfs_grid": lambda: {"bfs_grid4096": bfs_grid_row(stream)},
               "rmat16": lambda: {"rmat16": rmat16_row(stream, run)},
               "ppr": lambda: ppr_row(stream), "ppr_probe": lambda: ppr_probe_row(stream, 0),
               "ppr_probe_tile32": lambda: ppr_probe_row(stream, 32),
               "bfs_levels": lambda: bfs_levels_row(stream)}[args.row]()
        print(json.dumps(res), flush=True)
        return
    res, ctx = bench_tocab(args, world, rank, local)
    if rank == 0 and not args.quick:
        if not args.no_variants:
            res["variants"] = variants(args, ctx, world)
        res["e2e"] = e2e(args, ctx)
        if world == 1:
            res["cpu_baseline"] = cpu_baseline(ctx[0], args.cpu_seconds)
    if rank == 0:
        print(json.dumps(res), flush=True)
    barrier(world)


if __name__ == "__main__":
    main()
