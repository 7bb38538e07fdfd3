"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every expected value comes from a closed
form, an invariant, a textbook formulation computed a different way (dense Google matrix,
linear solve, Floyd-Warshall / scipy shortest paths) or brute force on tiny inputs.
"""
import itertools
import math

import numpy as np
import pytest

import graphgen as gg
import oracle

D = 0.85


def _pr(g, **kw):
    rp, ci = g.numpy()
    return oracle.pagerank_pull(g.V, rp, ci, **kw)


def _pr_push(g, **kw):
    rp, ci = g.numpy()
    return oracle.pagerank_push(g.V, rp, ci, **kw)


# ---------------------------------------------------------------- closed forms (Alg. 1/2)

@pytest.mark.parametrize("n", [1, 2, 3, 7, 64])
@pytest.mark.parametrize("iters", [0, 1, 5, 20])
def test_cycle_uniform(n, iters):
    if n == 1:
        g = gg.empty_graph(1)
    else:
        g = gg.cycle(n)
    for f in (_pr, _pr_push):
        r = f(g, iters=iters)
        np.testing.assert_allclose(r, np.full(n, 1.0 / n), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [2, 5, 16])
def test_complete_uniform(n):
    g = gg.complete(n)
    for f in (_pr, _pr_push):
        np.testing.assert_allclose(f(g, iters=20), np.full(n, 1.0 / n), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 17])
@pytest.mark.parametrize("d", [0.85, 0.5])
def test_star_closed_form(n, d):
    """Hub h and n leaves (edges both ways): h_k = h* + (-d)^k (1/V - h*),
    h* = (1 + d n) / ((n+1)(1+d)), leaves l_k = (1 - h_k)/n."""
    g = gg.star(n)
    V = n + 1
    hstar = (1 + d * n) / ((n + 1) * (1 + d))
    for k in [0, 1, 2, 3, 10, 20]:
        hk = hstar + (-d) ** k * (1.0 / V - hstar)
        lk = (1.0 - hk) / n
        for f in (_pr, _pr_push):
            r = f(g, iters=k, damping=d)
            assert abs(r[0] - hk) < 1e-14
            np.testing.assert_allclose(r[1:], lk, rtol=0, atol=1e-14)
    if n == 5 and d == 0.85:
        assert abs(_pr(g, iters=20)[0] - 0.4611006841723109) < 1e-15


@pytest.mark.parametrize("k", [0, 1, 2, 7, 20])
def test_two_vertices_dangling_redistribution(k):
    """Edge 0->1, vertex 1 dangling.  Redistributing D: r0* = 1/(2+d), and the error
    shrinks by -d/2 per step: r0_k = r0* + (-d/2)^k (1/2 - r0*); r1 = 1 - r0."""
    g = gg.from_edge_list(2, [(0, 1)])
    r0s = 1.0 / (2 + D)
    r0k = r0s + (-D / 2) ** k * (0.5 - r0s)
    for f in (_pr, _pr_push):
        r = f(g, iters=k)
        assert abs(r[0] - r0k) < 1e-15 and abs(r[1] - (1 - r0k)) < 1e-15
    # converged value
    r = _pr(g, iters=200)
    assert abs(r[0] - 1 / (2 + D)) < 1e-15 and abs(r[1] - (1 + D) / (2 + D)) < 1e-15


def test_two_vertices_drop_mode():
    """Literal Alg. 1 (no redistribution): r0 stays (1-d)/2, r1 = (1-d)/2 + d r0_prev."""
    g = gg.from_edge_list(2, [(0, 1)])
    r = _pr(g, iters=3, dangling="drop")
    assert abs(r[0] - (1 - D) / 2) < 1e-16
    assert abs(r[1] - ((1 - D) / 2 + D * (1 - D) / 2)) < 1e-16


# ---------------------------------------------------------------- invariants

def test_mass_conservation_and_drop_leak():
    g = gg.rmat(9, seed=5)
    rp, ci = g.numpy()
    deg = rp[1:] - rp[:-1]
    assert (deg == 0).any(), "want dangling vertices in this case"
    r = np.full(g.V, 1.0 / g.V)
    for _ in range(10):
        Dt = r[deg == 0].sum()
        rn = oracle.pagerank_pull(g.V, rp, ci, iters=1, dangling="drop", init=r)
        assert abs(rn.sum() - ((1 - D) + D * (1 - Dt))) < 1e-13
        rr = oracle.pagerank_pull(g.V, rp, ci, iters=1, init=r)
        assert abs(rr.sum() - 1.0) < 1e-13
        r = rr


def test_restart_from_init_equals_continuous_run():
    g = gg.rmat(9, seed=6)
    rp, ci = g.numpy()
    a = oracle.pagerank_pull(g.V, rp, ci, iters=20)
    h = oracle.pagerank_pull(g.V, rp, ci, iters=8)
    b = oracle.pagerank_pull(g.V, rp, ci, iters=12, init=h)
    np.testing.assert_array_equal(a, b)


def test_thread_count_does_not_change_result():
    g = gg.rmat(12, seed=8)
    rp, ci = g.numpy()
    a = oracle.pagerank_pull(g.V, rp, ci, nthreads=1)
    b = oracle.pagerank_pull(g.V, rp, ci, nthreads=4)
    np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------- textbook formulation

def _google_matrix(V, rp, ci, d, redistribute=True):
    """Dense column-stochastic M (M[v,u] = 1/outdeg(u) for u->v; dangling columns 1/V
    when redistributing), Google matrix G = d*M + (1-d)/V."""
    M = np.zeros((V, V))
    for u in range(V):
        deg = rp[u + 1] - rp[u]
        if deg == 0:
            if redistribute:
                M[:, u] = 1.0 / V
            continue
        for e in range(rp[u], rp[u + 1]):
            M[ci[e], u] += 1.0 / deg
    return d * M + (1 - d) / V, M


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("mode", ["redistribute", "drop"])
def test_dense_power_iteration(seed, mode):
    V = 200
    g = gg.random_small(V, 700, seed=seed)  # sparse enough to have dangling vertices
    rp, ci = g.numpy()
    assert ((rp[1:] - rp[:-1]) == 0).any()
    Gm, M = _google_matrix(V, rp, ci, D, redistribute=(mode == "redistribute"))
    x = np.full(V, 1.0 / V)
    for _ in range(20):
        # mass is conserved when redistributing, so the Google matrix applies as is;
        # dropping dangling mass makes the teleport term affine: d M x + (1-d)/V
        x = Gm @ x if mode == "redistribute" else D * (M @ x) + (1 - D) / V
    np.testing.assert_allclose(_pr(g, dangling=mode), x, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(_pr_push(g, dangling=mode), x, rtol=1e-12, atol=1e-16)


def test_linear_solve_at_convergence():
    V = 150
    g = gg.random_small(V, 600, seed=9)
    rp, ci = g.numpy()
    _, M = _google_matrix(V, rp, ci, D)
    x = np.linalg.solve(np.eye(V) - D * M, np.full(V, (1 - D) / V))
    np.testing.assert_allclose(_pr(g, iters=300), x, rtol=1e-12, atol=0)


def test_pull_equals_push_on_rmat():
    g = gg.rmat(11, seed=4)
    np.testing.assert_allclose(_pr(g), _pr_push(g), rtol=1e-12, atol=0)


# ---------------------------------------------------------------- transpose / partition

def test_transpose_bruteforce():
    g = gg.random_small(300, 2000, seed=12)
    rp, ci = g.numpy()
    trp, tci = oracle.transpose(g.V, rp, ci)
    edges = sorted((int(v), u) for u in range(g.V) for v in ci[rp[u]:rp[u + 1]])
    got = [(v, int(tci[e])) for v in range(g.V) for e in range(trp[v], trp[v + 1])]
    assert got == edges


@pytest.mark.parametrize("W", [1, 7, 64, 100, 299, 300, 1000])
def test_partition_bruteforce(W):
    V = 300
    g = gg.random_small(V, 2500, seed=21)
    trp, tci = oracle.transpose(V, *g.numpy())
    p = oracle.partition(V, trp, tci, W)
    B = math.ceil(V / W)
    assert p["B"] == B
    all_edges = {(v, int(tci[e])) for v in range(V) for e in range(trp[v], trp[v + 1])}
    seen = set()
    for b in range(B):
        lo, hi = b * W, min((b + 1) * W, V)
        want_rows = sorted({v for (v, u) in all_edges if lo <= u < hi})
        r0, r1 = p["blk_rows"][b], p["blk_rows"][b + 1]
        assert list(p["id_map"][r0:r1]) == want_rows          # local IDs ascending
        for r in range(r0, r1):
            v = int(p["id_map"][r])
            cols = [int(c) for c in p["colidx"][p["rowptr"][r]:p["rowptr"][r + 1]]]
            assert len(cols) >= 1
            assert cols == sorted(u for (vv, u) in all_edges if vv == v and lo <= u < hi)
            seen.update((v, u) for u in cols)
        assert p["rowptr"][r0] == p["blk_edges"][b]
    assert seen == all_edges and p["blk_edges"][-1] == len(all_edges)


def test_partition_block_sums_reproduce_pull():
    """Alg. 4 + merge: summing per-block partial sums gives Alg. 1's sums."""
    g = gg.rmat(10, seed=31)
    rp, ci = g.numpy()
    V = g.V
    trp, tci = oracle.transpose(V, rp, ci)
    deg = (rp[1:] - rp[:-1]).astype(np.float64)
    x = np.random.default_rng(0).random(V)
    want = np.array([x[tci[trp[v]:trp[v + 1]]].sum() for v in range(V)])
    p = oracle.partition(V, trp, tci, 97)
    got = np.zeros(V)
    for r in range(len(p["id_map"])):
        got[p["id_map"][r]] += x[p["colidx"][p["rowptr"][r]:p["rowptr"][r + 1]]].sum()
    np.testing.assert_allclose(got, want, rtol=1e-12)
    del deg


def test_table3_block_width_reading():
    """256 Ki source vertices per subgraph reproduces Table 3 within V's print rounding."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_subgraphs.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 8
    for name, vp, unit, cnt in rows:
        vp, unit, cnt = float(vp), float(unit), int(cnt)
        lo, hi = vp - unit / 2, vp + unit / 2
        # some V in [lo, hi] with ceil(V / 262144) == cnt  <=>  intervals overlap
        assert (cnt - 1) * 262144 < hi and cnt * 262144 >= lo, name
        # and the neighbouring widths do not fit every row
    assert not all(math.ceil(float(r[1]) / 131072) == int(r[3]) for r in rows)


# ---------------------------------------------------------------- BFS

def _bfs(g, s):
    rp, ci = g.numpy()
    return oracle.bfs(g.V, rp, ci, s)


@pytest.mark.parametrize("n,s", [(1, 0), (2, 1), (10, 0), (10, 4), (257, 100)])
def test_bfs_path(n, s):
    g = gg.path(n) if n > 1 else gg.empty_graph(1)
    np.testing.assert_array_equal(_bfs(g, s), np.abs(np.arange(n) - s))


def test_bfs_directed_path_unreachable():
    g = gg.path(6, directed=True)
    np.testing.assert_array_equal(_bfs(g, 2), [-1, -1, 0, 1, 2, 3])


def test_bfs_grid_manhattan():
    R, C = 13, 17
    g = gg.grid2d(R, C, drop=0.0)
    s = 5 * C + 9
    lv = _bfs(g, s)
    want = np.array([abs(i // C - 5) + abs(i % C - 9) for i in range(R * C)])
    np.testing.assert_array_equal(lv, want)


def test_bfs_complete_and_disconnected():
    np.testing.assert_array_equal(_bfs(gg.complete(6), 3), [1, 1, 1, 0, 1, 1])
    g = gg.from_edge_list(6, [(0, 1), (1, 0), (2, 3), (3, 2), (4, 5)])
    np.testing.assert_array_equal(_bfs(g, 0), [0, 1, -1, -1, -1, -1])
    np.testing.assert_array_equal(_bfs(g, 4), [-1, -1, -1, -1, 0, 1])


@pytest.mark.parametrize("seed", [3, 4])
def test_bfs_vs_floyd_warshall(seed):
    scipy_sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    V = 180
    g = gg.random_small(V, 400, seed=seed)
    rp, ci = g.numpy()
    A = scipy_sp.csr_matrix((np.ones(ci.size), ci, rp), shape=(V, V))
    dist = csgraph.shortest_path(A, method="FW", unweighted=True)
    for s in [0, 17, 99]:
        want = np.where(np.isinf(dist[s]), -1, dist[s]).astype(np.int64)
        np.testing.assert_array_equal(_bfs(g, s), want)


def test_bfs_boolean_powers():
    """Level L set = vertices reached by a walk of length L and not of any shorter length."""
    V = 40
    g = gg.random_small(V, 70, seed=77)
    rp, ci = g.numpy()
    A = np.zeros((V, V), dtype=bool)
    for u in range(V):
        A[u, ci[rp[u]:rp[u + 1]]] = True
    s = 0
    want = np.full(V, -1)
    reach = np.zeros(V, bool)
    reach[s] = True
    want[s] = 0
    cur = reach.copy()
    for L in range(1, V):
        cur = (cur.astype(int) @ A.astype(int)) > 0
        new = cur & ~reach
        want[new] = L
        reach |= cur
    np.testing.assert_array_equal(_bfs(g, s), want)


# ---------------------------------------------------------------- personalised PageRank

def test_ppr_linear_solve():
    V = 120
    g = gg.random_small(V, 500, seed=41)
    rp, ci = g.numpy()
    _, M0 = _google_matrix(V, rp, ci, D, redistribute=False)
    dang = (rp[1:] - rp[:-1]) == 0
    srcs = [0, 5, 77]
    R = oracle.ppr_pull(V, rp, ci, srcs, iters=400)
    for j, s in enumerate(srcs):
        # x = d M0 x + (d * sum_dangling(x) + (1-d)) e_s
        A = np.eye(V) - D * M0
        A[s, dang] -= D
        rhs = np.zeros(V)
        rhs[s] = 1 - D
        np.testing.assert_allclose(R[:, j], np.linalg.solve(A, rhs), rtol=1e-11, atol=1e-15)
        assert abs(R[:, j].sum() - 1) < 1e-12


def test_ppr_average_is_global_pagerank_without_dangling():
    """With no dangling vertex, the mean of the V personalised vectors (teleport to s,
    start at e_s) equals global PageRank (teleport uniform, start 1/V), every iteration."""
    g = gg.grid2d(6, 7, drop=0.0)
    rp, ci = g.numpy()
    V = g.V
    for iters in (1, 3, 20):
        R = oracle.ppr_pull(V, rp, ci, list(range(V)), iters=iters)
        np.testing.assert_allclose(R.mean(axis=1), _pr(g, iters=iters), rtol=1e-12)


def test_ppr_zero_damping_is_teleport():
    g = gg.rmat(7, seed=2)
    rp, ci = g.numpy()
    R = oracle.ppr_pull(g.V, rp, ci, [3, 9], damping=0.0, iters=5)
    want = np.zeros((g.V, 2))
    want[3, 0] = 1
    want[9, 1] = 1
    np.testing.assert_array_equal(R, want)


# ---------------------------------------------------------------- MLP oracle

def _params(rng, H=12, scale=0.3):
    return {"W1": rng.normal(0, scale, (16, 64)), "b1": rng.normal(0, 0.1, 64),
            "W2": rng.normal(0, scale, (64, 64)), "b2": rng.normal(0, 0.1, 64),
            "W3": rng.normal(0, scale, (64, H)), "b3": rng.normal(0, 0.1, H)}


def test_mlp_zero_weights_loss():
    heads = (7, 3, 2)
    p = {k: np.zeros_like(v) for k, v in _params(np.random.default_rng(0)).items()}
    x = np.random.default_rng(1).normal(size=(5, 16))
    y = np.array([[0, 1, 1], [6, 2, 0], [3, 0, 1], [1, 1, 0], [2, 2, 1]])
    assert abs(oracle.mlp_loss(p, x, y, heads) - (math.log(7) + math.log(3) + math.log(2))) < 1e-14


def test_mlp_gradients_finite_differences():
    heads = (7, 3, 2)
    rng = np.random.default_rng(3)
    p = _params(rng)
    x = rng.normal(size=(9, 16))
    y = np.stack([rng.integers(0, h, 9) for h in heads], axis=1)
    g = oracle.mlp_backward(p, x, y, heads)
    h = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = oracle.mlp_loss(p, x, y, heads)
            flat[idx] = old - h
            lm = oracle.mlp_loss(p, x, y, heads)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - g[k].reshape(-1)[idx]) < 1e-7 * max(1.0, abs(num)), (k, idx)


def test_adam_first_step_is_signed_lr():
    from oracle.mlp import adam_step
    p = {"w": np.array([1.0, -2.0, 3.0])}
    gr = {"w": np.array([0.5, -4.0, 1e-3])}
    z = {"w": np.zeros(3)}
    newp, m, v = adam_step(p, gr, z, z, t=1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(newp["w"], p["w"] - 0.01 * np.sign(gr["w"]), rtol=1e-15)
