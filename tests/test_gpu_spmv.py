"""SpMV through the C ABI against the FP64 oracle.  The GPU sums in FP32 (fused multiply-adds per
lane, then a 5-level shuffle tree), so row i may differ from the exact product by at most
(d_i + 6) * 2^-24 * sum_k |a_ik x_k| (d_i = stored entries of the row): the standard bound for a
summation whose longest chain has at most d_i + 5 roundings.  The inputs are the same FP32 values
on both sides."""
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


def _check(T, g, vals, x):
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    y = T.spmv(G, vals.cuda(), x.cuda()).cpu().numpy().astype(np.float64)
    rp, ci = g.numpy()
    v64, x64 = vals.numpy().astype(np.float64), x.numpy().astype(np.float64)
    want = oracle.spmv(g.V, rp, ci, v64, x64)
    mag = oracle.spmv(g.V, rp, ci, np.abs(v64), np.abs(x64))
    bound = (np.diff(rp) + 6) * 2.0 ** -24 * mag
    assert np.all(np.abs(y - want) <= bound + 1e-30)
    again = T.spmv(G, vals.cuda(), x.cuda()).cpu().numpy().astype(np.float64)
    assert np.array_equal(y, again)  # fixed reduction order
    return y


@pytest.mark.parametrize("name", ["rmat", "er", "plc", "grid"])
def test_matches_oracle_within_the_fp32_bound(T, name):
    g = {"rmat": gg.rmat(12), "er": gg.random_small(3000, 40000, 2), "plc": gg.powerlaw_config(4000, 8, 2.2, seed=5),
         "grid": gg.grid2d(60, 70)}[name]
    vals = gg.edge_values(g, seed=31)
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(g.V).astype(np.float32))
    _check(T, g, vals, x)


def test_hub_rows_and_empty_rows(T):
    g = gg.star(5000)  # one row of 5,000 entries, 5,000 rows of one
    vals = gg.edge_values(g, seed=2)
    x = torch.ones(g.V, dtype=torch.float32)
    _check(T, g, vals, x)
    e = gg.empty_graph(100)
    y = _check(T, e, torch.zeros(0, dtype=torch.float32), torch.ones(100, dtype=torch.float32))
    assert np.all(y == 0.0)


def test_identity_permutation_exact(T):
    n = 1000
    perm = torch.from_numpy(np.random.default_rng(4).permutation(n).astype(np.int32))
    rp = torch.arange(n + 1, dtype=torch.int32)  # row i holds one entry, at column perm[i]
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(n).astype(np.float32))
    G = T.graph_load_csr(rp.cuda(), perm.cuda(), V=n)
    y = T.spmv(G, torch.ones(n, dtype=torch.float32, device="cuda"), x.cuda()).cpu()
    assert torch.equal(y, x[perm.long()])
    y = T.spmv(G, torch.full((n,), 2.0, device="cuda"), x.cuda()).cpu()
    assert torch.equal(y, 2.0 * x[perm.long()])


def test_host_memory_is_refused(T):
    g = gg.path(4)
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    from paper_1904_02241_gb300 import _lib as L
    v = torch.ones(g.E, dtype=torch.float32)  # host buffers: refused before any access
    x = torch.ones(g.V, dtype=torch.float32)
    st = L.load().tc_spmv(G.handle, v.data_ptr(), x.data_ptr(), x.data_ptr(), L.TC_MEM_HOST, None)
    assert st == -6


# ------------------------------------------------------------------ GC-pull SpMV (TOCAB, value stream)

@pytest.mark.parametrize("name", ["rmat", "er", "plc", "grid", "star"])
@pytest.mark.parametrize("B", [1, 3, 8, 64])
def test_gc_pull_matches_oracle_within_the_fp32_bound(T, name, B):
    """The pieces of a row are summed like a row of the warp form, then added in block order: at
    most d_i + 6 + B roundings in the longest chain."""
    g = {"rmat": gg.rmat(12), "er": gg.random_small(3000, 40000, 2), "plc": gg.powerlaw_config(4000, 8, 2.2, seed=5),
         "grid": gg.grid2d(60, 70), "star": gg.star(5000)}[name]
    if B > g.V:
        pytest.skip("B > V")
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    P = T.tocab_partition(G, T.TC_PUSH, B, merge_range=1024)
    vals = gg.edge_values(g, seed=31)
    x = torch.from_numpy(np.random.default_rng(B).standard_normal(g.V).astype(np.float32))
    T.part_set_values(P, vals.cuda())
    y = T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64)
    rp, ci = g.numpy()
    v64, x64 = vals.numpy().astype(np.float64), x.numpy().astype(np.float64)
    want = oracle.spmv(g.V, rp, ci, v64, x64)
    mag = oracle.spmv(g.V, rp, ci, np.abs(v64), np.abs(x64))
    bound = (np.diff(rp) + 6 + P.num_blocks) * 2.0 ** -24 * mag
    assert np.all(np.abs(y - want) <= bound + 1e-30)
    assert np.array_equal(y, T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64))  # fixed order
    # new values through the same partition (the recorded entry order is reused)
    vals2 = gg.edge_values(g, seed=32)
    T.part_set_values(P, vals2.cuda())
    y2 = T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64)
    v2 = vals2.numpy().astype(np.float64)
    want2 = oracle.spmv(g.V, rp, ci, v2, x64)
    bound2 = (np.diff(rp) + 6 + P.num_blocks) * 2.0 ** -24 * oracle.spmv(g.V, rp, ci, np.abs(v2), np.abs(x64))
    assert np.all(np.abs(y2 - want2) <= bound2 + 1e-30)


def test_gc_pull_permutation_matrix_is_exact(T):
    n = 3000
    perm = np.random.default_rng(9).permutation(n)
    g = gg.from_edge_list(n, np.stack([np.arange(n), perm], 1))
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=n)
    P = T.tocab_partition(G, T.TC_PUSH, 7, merge_range=512)
    T.part_set_values(P, torch.ones(g.E, dtype=torch.float32, device="cuda"))
    x = torch.from_numpy(np.random.default_rng(1).standard_normal(n).astype(np.float32)).cuda()
    y = T.spmv_tocab(P, x).cpu().numpy()
    rp, ci = g.numpy()
    want = np.zeros(n, np.float32)  # rows whose entry was a self loop were dropped: they are empty
    want[np.repeat(np.arange(n), np.diff(rp))] = x.cpu().numpy()[ci]
    np.testing.assert_array_equal(y, want)  # row i holds x[perm[i]] exactly


def test_gc_pull_refusals(T):
    g = gg.rmat(10)
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    x = torch.ones(g.V, dtype=torch.float32, device="cuda")
    Pr = T.tocab_partition(G, T.TC_PULL, 2, order="outdegree")
    with pytest.raises(T.TocabError):
        T.part_set_values(Pr, torch.ones(g.E, dtype=torch.float32, device="cuda"))  # renumbered
    for d in (T.TC_PUSH, T.TC_PULL):
        P = T.tocab_partition(G, d, 2)
        with pytest.raises(T.TocabError):
            T.spmv_tocab(P, x)  # no values yet


# ------------------------------------------------------------------ GC-push SpMV (TOCAB, atomics)

@pytest.mark.parametrize("name", ["rmat", "er", "plc", "grid", "star"])
@pytest.mark.parametrize("B", [1, 3, 8, 64])
def test_gc_push_matches_oracle_within_the_fp32_bound(T, name, B):
    """Row i gets one rounded product per entry added by FP32 atomics in some order: at most
    d_i + 1 roundings in the longest chain, whatever the order (bound taken with d_i + 6)."""
    g = {"rmat": gg.rmat(12), "er": gg.random_small(3000, 40000, 2), "plc": gg.powerlaw_config(4000, 8, 2.2, seed=5),
         "grid": gg.grid2d(60, 70), "star": gg.star(5000)}[name]
    if B > g.V:
        pytest.skip("B > V")
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    P = T.tocab_partition(G, T.TC_PULL, B)
    vals = gg.edge_values(g, seed=41)
    x = torch.from_numpy(np.random.default_rng(B + 7).standard_normal(g.V).astype(np.float32))
    T.part_set_values(P, vals.cuda())
    rp, ci = g.numpy()
    v64, x64 = vals.numpy().astype(np.float64), x.numpy().astype(np.float64)
    want = oracle.spmv(g.V, rp, ci, v64, x64)
    bound = (np.diff(rp) + 6) * 2.0 ** -24 * oracle.spmv(g.V, rp, ci, np.abs(v64), np.abs(x64))
    for _ in range(2):  # every call within the bound (the addition order may differ)
        y = T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64)
        assert np.all(np.abs(y - want) <= bound + 1e-30)
    # new values through the same partition
    vals2 = gg.edge_values(g, seed=42)
    T.part_set_values(P, vals2.cuda())
    v2 = vals2.numpy().astype(np.float64)
    y2 = T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64)
    bound2 = (np.diff(rp) + 6) * 2.0 ** -24 * oracle.spmv(g.V, rp, ci, np.abs(v2), np.abs(x64))
    assert np.all(np.abs(y2 - oracle.spmv(g.V, rp, ci, v2, x64)) <= bound2 + 1e-30)


def test_gc_push_permutation_matrix_is_exact(T):
    """One entry per row: each y[i] is one product with nothing to add, so exact, and it checks
    the value order of the pull partition (transpose, then blocks)."""
    n = 3000
    perm = np.random.default_rng(10).permutation(n)
    g = gg.from_edge_list(n, np.stack([np.arange(n), perm], 1))
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=n)
    P = T.tocab_partition(G, T.TC_PULL, 7)
    vals = torch.from_numpy(np.random.default_rng(2).standard_normal(g.E).astype(np.float32))
    T.part_set_values(P, vals.cuda())
    x = torch.from_numpy(np.random.default_rng(3).standard_normal(n).astype(np.float32)).cuda()
    y = T.spmv_tocab(P, x).cpu().numpy()
    rp, ci = g.numpy()
    want = np.zeros(n, np.float32)  # rows whose entry was a self loop were dropped: they are empty
    want[np.repeat(np.arange(n), np.diff(rp))] = vals.numpy() * x.cpu().numpy()[ci]
    np.testing.assert_array_equal(y, want)


def test_gc_push_agrees_with_gc_pull_and_vwc_on_rmat16(T):
    """The three SpMV forms on one matrix: each within the FP32 bound of the FP64 product."""
    g = gg.rmat(16)
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
    vals = gg.edge_values(g, seed=5)
    x = torch.from_numpy(np.random.default_rng(5).standard_normal(g.V).astype(np.float32))
    rp, ci = g.numpy()
    v64, x64 = vals.numpy().astype(np.float64), x.numpy().astype(np.float64)
    want = oracle.spmv(g.V, rp, ci, v64, x64)
    mag = oracle.spmv(g.V, rp, ci, np.abs(v64), np.abs(x64))
    Ppull = T.tocab_partition(G, T.TC_PUSH, 8)
    Ppush = T.tocab_partition(G, T.TC_PULL, 8)
    T.part_set_values(Ppull, vals.cuda())
    T.part_set_values(Ppush, vals.cuda())
    for y, extra in ((T.spmv(G, vals.cuda(), x.cuda()), 0), (T.spmv_tocab(Ppull, x.cuda()), 8),
                     (T.spmv_tocab(Ppush, x.cuda()), 0)):
        err = np.abs(y.cpu().numpy().astype(np.float64) - want)
        assert np.all(err <= (np.diff(rp) + 6 + extra) * 2.0 ** -24 * mag + 1e-30)


@pytest.mark.parametrize("d", ["push", "pull"])
def test_tocab_spmv_on_degenerate_matrices(T, d):
    """No stored entries (y = 0) and a single entry, through both partition directions."""
    direction = T.TC_PUSH if d == "push" else T.TC_PULL
    for g in (gg.empty_graph(5), gg.from_edge_list(3, [(2, 0)])):
        G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)
        P = T.tocab_partition(G, direction, 1)
        vals = torch.full((g.E,), 1.5, dtype=torch.float32, device="cuda")
        T.part_set_values(P, vals)
        x = torch.arange(1, g.V + 1, dtype=torch.float32, device="cuda")
        y = T.spmv_tocab(P, x).cpu().numpy()
        want = np.zeros(g.V, np.float32)
        if g.E:
            want[2] = 1.5 * 1.0  # row 2 holds one entry in column 0
        np.testing.assert_array_equal(y, want)
