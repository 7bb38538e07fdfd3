"""Betweenness centrality through the C ABI against the FP64 oracle: Alg. 3's depths and
shortest-path counts exactly, the scores within rounding of the oracle's, on graphs with
branching shortest paths (grids, hypercubes), skew (R-MAT), directed reachability gaps,
isolated vertices and no edges."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_02241_gb300 as T
    T.lib()
    return T


def _hypercube(k):
    return gg.from_edge_list(1 << k, [(x, x ^ (1 << b)) for x in range(1 << k) for b in range(k)])


GRAPHS = {
    "path": gg.path(40),
    "dpath": gg.path(30, directed=True),
    "star": gg.star(50),
    "grid": gg.grid2d(12, 15, drop=0.0),
    "grid_drop": gg.grid2d(20, 20, drop=0.2, seed=3),
    "cube": _hypercube(7),
    "rmat": gg.symmetrize(gg.rmat(9)),
    "rmat_dir": gg.rmat(9, seed=4),
    "er": gg.random_small(300, 1400, 6),
    "empty": gg.empty_graph(9),
}
# hubs with hundreds of in-edges (warp-per-row pull levels) beside small frontiers (push levels);
# checked from a few sources only
BIG = {
    "rmat13_sym": gg.symmetrize(gg.rmat(13)),
    "big_star": gg.symmetrize(gg.star(3000)),
}


def _load(T, g):
    return T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_forward_depths_and_counts_exact(T, name):
    g = GRAPHS[name]
    G = _load(T, g)
    rp, ci = g.numpy()
    for s in sorted({0, g.V // 2, g.V - 1}):
        depth, sigma = T.bc_forward(G, s)
        want_d, want_s = oracle.bc_forward(g.V, rp, ci, s)
        assert np.array_equal(depth.cpu().numpy(), want_d), (name, s)
        assert np.array_equal(sigma.cpu().numpy(), want_s), (name, s)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_scores_all_sources(T, name):
    g = GRAPHS[name]
    G = _load(T, g)
    rp, ci = g.numpy()
    got = T.bc(G).cpu().numpy()
    want = oracle.bc(g.V, rp, ci)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-9)
    assert torch.equal(T.bc(G).cpu(), torch.from_numpy(got))  # deterministic


def test_scores_source_subset_and_host_output(T):
    g = gg.symmetrize(gg.rmat(12))
    G = _load(T, g)
    rp, ci = g.numpy()
    srcs = gg.sources(g, 8, seed=13)
    want = oracle.bc(g.V, rp, ci, srcs)
    dev = T.bc(G, srcs).cpu().numpy()
    np.testing.assert_allclose(dev, want, rtol=1e-12, atol=1e-9)
    host = torch.empty(g.V, dtype=torch.float64)
    T.bc(G, srcs, out=host)
    assert np.array_equal(host.numpy(), dev)
    assert np.all(T.bc(G, []).cpu().numpy() == 0.0)


def test_closed_forms_on_device(T):
    n = 25
    G = _load(T, gg.path(n))
    assert np.array_equal(T.bc(G).cpu().numpy(), np.array([2.0 * i * (n - 1 - i) for i in range(n)]))
    G = _load(T, gg.star(30))
    s = T.bc(G).cpu().numpy()
    assert s[0] == 30 * 29 and np.all(s[1:] == 0.0)


@pytest.mark.parametrize("n", [64, 65, 2048, 2049])
def test_star_hub_at_each_degree_class(T, n):
    """The backward sweep sums a vertex's children in one of three kernels chosen by out-degree
    (8 lanes up to 64, a warp up to the hub degree 2048, a CTA above): stars whose hub sits on
    each side of both boundaries give the closed form n (n - 1) for the hub and 0 for the leaves."""
    G = _load(T, gg.star(n))
    s = T.bc(G).cpu().numpy()
    assert s[0] == float(n * (n - 1)) and np.all(s[1:] == 0.0)


def test_invalid_source_is_refused(T):
    G = _load(T, gg.path(5))
    with pytest.raises(T.TocabError) as e:
        T.bc(G, [7])
    assert e.value.status == -1
    with pytest.raises(T.TocabError):
        T.bc_forward(G, -1)


@pytest.mark.parametrize("name", ["rmat13_sym", "big_star", "grid", "dpath"])
def test_scores_repeat_bit_for_bit(T, name):
    """Push levels (FP64 atomics on integer path counts) and warp trees leave no trace of timing;
    depths and counts stay exact."""
    g = BIG[name] if name in BIG else GRAPHS[name]
    G = _load(T, g)
    srcs = [0, g.V // 3, g.V - 1]
    a = T.bc(G, srcs).cpu()
    assert torch.equal(a, T.bc(G, srcs).cpu())
    rp, ci = g.numpy()
    np.testing.assert_allclose(a.numpy(), oracle.bc(g.V, rp, ci, srcs), rtol=1e-12, atol=1e-9)
    for s in srcs:
        depth, sigma = T.bc_forward(G, s)
        want_d, want_s = oracle.bc_forward(g.V, rp, ci, s)
        assert np.array_equal(depth.cpu().numpy(), want_d)
        assert np.array_equal(sigma.cpu().numpy(), want_s)


@pytest.mark.parametrize("name", ["rmat13_sym", "big_star", "grid", "rmat", "rmat_dir", "er", "dpath", "empty"])
@pytest.mark.parametrize("B", [1, 4, 16])
def test_blocked_pull_levels_give_the_same_bits(T, name, B):
    """tc_bc_tocab (TOCAB pull levels, sigma sums merged in block order) against tc_bc: the path
    counts are integers, so depths, sigma and the scores must agree bit for bit; and both against
    the oracle."""
    g = BIG[name] if name in BIG else GRAPHS[name]
    if B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, merge_range=1024, smem_stage=-1)
    srcs = [0, g.V // 3, g.V - 1]
    a = T.bc(G, srcs).cpu()
    b = T.bc(G, srcs, part=P).cpu()
    assert torch.equal(a, b)
    rp, ci = g.numpy()
    np.testing.assert_allclose(b.numpy(), oracle.bc(g.V, rp, ci, srcs), rtol=1e-12, atol=1e-9)


def test_blocked_bc_refuses_other_partitions(T):
    g = GRAPHS["rmat"]
    G = _load(T, g)
    with pytest.raises(T.TocabError):
        T.bc(G, [0], part=T.tocab_partition(G, T.TC_PUSH, 2))
    with pytest.raises(T.TocabError):
        T.bc(G, [0], part=T.tocab_partition(G, T.TC_PULL, 2, order="outdegree"))
