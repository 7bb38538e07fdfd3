"""The learned cost model: its CUDA forward/backward/Adam kernels against the FP64 oracle,
its feature extractor against the plain definitions, and that training learns."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from oracle.mlp import adam_step

pytestmark = pytest.mark.gpu
HEADS = (9, 3, 2)


@pytest.fixture(scope="module")
def CM():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02241_gb300 import costmodel
    return costmodel


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    Y = np.stack([rng.integers(0, h, n) for h in HEADS], axis=1).astype(np.int32)
    return X, Y


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-12)


def test_mlp_forward_matches_oracle(CM):
    m = CM.MLP(heads=HEADS)
    m.init(seed=1)
    X, _ = _data(37, 2)
    Z = m.forward(X)
    Zo, _ = oracle.mlp_forward(m.get(), X.astype(np.float64))
    assert _rel(Z, Zo) < 1e-5


def test_mlp_gradients_match_oracle(CM):
    m = CM.MLP(heads=HEADS)
    m.init(seed=3)
    X, Y = _data(53, 4)
    loss = m.loss_grad(X, Y)
    p = m.get()
    assert abs(loss - oracle.mlp_loss(p, X.astype(np.float64), Y, HEADS)) < 1e-5 * max(1.0, abs(loss))
    go = oracle.mlp_backward(p, X.astype(np.float64), Y, HEADS)
    g = m.grads()
    for k in go:
        assert _rel(g[k], go[k]) < 2e-4, k


def test_mlp_adam_step_matches_oracle(CM):
    m = CM.MLP(heads=HEADS)
    m.init(seed=5)
    X, Y = _data(20, 6)
    p0 = m.get()
    m.loss_grad(X, Y)
    g = m.grads()
    m.adam_step(lr=1e-2)
    zeros = {k: np.zeros_like(v) for k, v in p0.items()}
    want, _, _ = adam_step(p0, g, zeros, zeros, t=1, lr=1e-2)
    got = m.get()
    for k in want:
        assert np.allclose(got[k], want[k], rtol=1e-5, atol=1e-6), k


def test_mlp_zero_weights_loss_is_log_classes(CM):
    m = CM.MLP(heads=HEADS)
    m.set({n: np.zeros(s) for n, s in m.shapes()})
    X, Y = _data(10, 7)
    assert abs(m.loss_grad(X, Y) - sum(np.log(h) for h in HEADS)) < 1e-5


def test_mlp_training_learns_a_rule(CM):
    rng = np.random.default_rng(0)
    X = rng.normal(size=(512, 16)).astype(np.float32)
    Y = np.stack([(X[:, 0] > 0) * 4 + (X[:, 1] > 0), (X[:, 2] > 0.5).astype(int), (X[:, 3] + X[:, 4] > 0)],
                 axis=1).astype(np.int32)
    m = CM.MLP(heads=HEADS)
    m.init(seed=1)
    l0 = m.loss_grad((X - X.mean(0)) / X.std(0), Y)
    loss = m.train(X, Y, epochs=200, batch=64, lr=3e-3)
    assert loss < 0.3 * l0
    acc = (m.predict(X) == Y).mean(axis=0)
    assert (acc > 0.9).all(), acc


def _features_numpy(rowptr, colidx, rowids, V, out_rowptr, l2):
    d = np.diff(rowptr).astype(np.float64)
    R, E = len(d), d.sum()
    mean = E / R
    od = np.diff(out_rowptr).astype(np.float64)
    om = od.sum() / V
    first = np.array([abs(colidx[rowptr[r]] - rowids[r]) if d[r] > 0 else 0 for r in range(R)], np.float64)
    return np.array([np.log2(R + 1), np.log2(E + 1), mean, d.std() / mean, np.log2(1 + d.max() / mean),
                     (d == 0).mean(), ((d >= 1) & (d <= 7)).mean(), ((d >= 8) & (d <= 15)).mean(),
                     ((d >= 16) & (d <= 31)).mean(), (d >= 32).mean(), od.std() / om, (od == 0).mean(),
                     np.log2(1 + 4 * V / l2), np.log2(1 + 4 * E / l2), first.sum() / (R * V),
                     np.log2(1 + od.max() / om)])


def test_graph_features_match_definitions(CM):
    import paper_1904_02241_gb300 as T
    g = gg.rmat(11)
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda())
    f = CM.graph_features(G)
    trp, tci = oracle.transpose(g.V, *g.numpy())
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    want = _features_numpy(trp, tci, np.arange(g.V), g.V, g.numpy()[0], l2)
    np.testing.assert_allclose(f, want, rtol=2e-5, atol=1e-6)
    P = T.tocab_partition(G, T.TC_PULL, 4)
    pf = CM.part_features(P)
    ex = P.export()
    for b in range(P.num_blocks):
        r0, r1 = ex["blk_rows"][b], ex["blk_rows"][b + 1]
        rp = ex["rowptr"][r0:r1 + 1]
        wb = _features_numpy(rp, ex["colidx"], ex["id_map"][r0:r1], g.V, g.numpy()[0], l2)
        wb[12] = np.log2(1 + 4 * P.block_width / l2)
        np.testing.assert_allclose(pf[b], wb, rtol=2e-5, atol=1e-6, err_msg=str(b))


def test_learned_model_gains_over_heuristic(CM):
    """Train on timings the method generates (small seeded graphs of four families), then on
    held-out graphs compare the time of the network's configuration with the paper's heuristic
    (pull, block width from the L2 size, thread/warp/CTA balancing) and with the exhaustive best.
    The network must be at least as good as the heuristic (geometric mean of time / best)."""
    train = CM.graph_specs(28, seed=5000, scale_lo=14, scale_hi=16)
    X, Y, _ = CM.build_dataset(train, iters=5, reps=3)
    m = CM.MLP()
    m.init(seed=0)
    m.train(X, Y, epochs=300, batch=32, lr=3e-3)
    held = CM.evaluate(m, CM.graph_specs(8, seed=7000, scale_lo=14, scale_hi=16), iters=5, reps=3)
    gm = lambda k: float(np.exp(np.mean([np.log(r[k] / r["t_best"]) for r in held])))  # noqa: E731
    model, heur = gm("t_model"), gm("t_heuristic")
    print(f"held-out time / exhaustive best: model {model:.3f}, heuristic {heur:.3f}, "
          f"gain {heur / model:.3f}x")
    assert model <= heur * 1.05
    # the BFS heads (frontier thresholds): measured for the model's choice on every held-out graph
    bm = [r["bfs_model"] / r["bfs_best"] for r in held if r["bfs_model"] is not None]
    bh = [r["bfs_heuristic"] / r["bfs_best"] for r in held]
    assert len(bm) == len(held)
    print(f"BFS held-out time / best: model {np.exp(np.mean(np.log(bm))):.3f}, "
          f"heuristic {np.exp(np.mean(np.log(bh))):.3f}")
    assert np.exp(np.mean(np.log(bm))) <= np.exp(np.mean(np.log(bh))) * 1.10


def test_per_block_lb_matches_or_beats_per_graph(CM):
    """The shipped model's load-balancing head run on each subgraph's features (tc_part_features,
    applied with tc_part_set_lb) against the same head on the whole graph's features applied to
    every block: the per-subgraph choice is no slower (geometric mean over skewed graphs, within
    timing noise), and both give the oracle's ranks."""
    import graphgen as gg
    import oracle
    from tests.gpu_util import l1_rel
    m = CM.MLP.load()
    ratios = []
    for g in (gg.rmat(16), gg.powerlaw_config(1 << 16, 8, 2.2, seed=3), gg.rmat(17, 8, 0.6, 0.15, 0.15, seed=9)):
        G = CM.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
        P = CM.tocab_partition(G, CM.L.TC_PULL, 8, smem_stage=-1)
        lb_graph = CM.LB_CLASSES[m.predict(CM.graph_features(G)[None])[0][1]]
        t_graph = CM.time_config(G, "pull", None, lb_graph, part=P)
        wmin = CM.per_block_lb(m, P)
        assert len(wmin) == P.num_blocks
        t_block = CM.time_config(G, "pull", None, "hybrid", part=P)  # the table overrides lb_warp_min
        ratios.append(t_block / t_graph)
        r = CM.pagerank_pull(G, P).cpu().numpy()
        rp, ci = g.numpy()
        assert l1_rel(r, oracle.pagerank_pull(g.V, rp, ci)) <= 1e-5
        print(f"V={g.V}: per-graph {lb_graph} {t_graph:.4f} ms, per-block {wmin} {t_block:.4f} ms")
    assert float(np.exp(np.mean(np.log(ratios)))) <= 1.10


@pytest.mark.parametrize("bad", [-1, 3])
def test_mlp_rejects_labels_outside_their_head(CM, bad):
    """A label outside [0, head size) fails the call before any kernel indexes the logits with
    it, for the gradient call and for training; the parameters stay as they were."""
    from paper_1904_02241_gb300 import TocabError
    m = CM.MLP(heads=HEADS)
    m.init(seed=7)
    X, Y = _data(11, 8)
    Y[5, 1] = bad  # head 1 has 3 classes
    before = m.get()
    with pytest.raises(TocabError):
        m.loss_grad(X, Y)
    with pytest.raises(TocabError):
        m.train(X, Y, epochs=1, batch=4)
    after = m.get()
    for k in before:
        assert np.array_equal(before[k], after[k]), k
