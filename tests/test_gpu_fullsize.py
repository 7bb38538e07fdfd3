"""Full-size parity: the workloads the benchmark times, in the launch configuration it times them
in, checked against the FP64 oracle on the host cores.  Every output is checked where the oracle
(OpenMP over destinations) finishes in seconds; PPR columns and the many-graph batch are checked
on a seeded sample.  Invariants (mass conservation, run-to-run identity) are checked beside.
The small configuration (R-MAT 16, unblocked and 4 source-range blocks) is checked in full."""
import os

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from gpu_util import l1_rel

pytestmark = pytest.mark.gpu
TOL = 1e-5
CORES = os.cpu_count() or 1


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_02241_gb300 as T
    T.lib()
    oracle.build()
    return T


def _load(T, g):
    return T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)


def test_rmat16_unblocked_and_four_blocks(T):
    """R-MAT 16 (V = 65,536, ~1M edges): unblocked pull and TOCAB with 4 source-range blocks."""
    g = gg.rmat(16)
    G = _load(T, g)
    rp, ci = g.numpy()
    want = oracle.pagerank_pull(g.V, rp, ci, nthreads=CORES)
    assert l1_rel(T.pagerank_pull(G, None).cpu().numpy(), want) <= TOL
    P = T.tocab_partition(G, T.TC_PULL, 4)
    assert P.num_blocks == 4
    assert l1_rel(T.pagerank_pull(G, P).cpu().numpy(), want) <= TOL
    assert l1_rel(T.pagerank_push(G, None).cpu().numpy(), want) <= TOL


@pytest.fixture(scope="module")
def rmat24(T):
    g = gg.rmat(24, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    rp, ci = g.numpy()
    tr = oracle.transpose(g.V, rp, ci)
    return g, G, rp, ci, tr


def test_rmat24_transpose_bit_exact(T, rmat24):
    g, G, rp, ci, tr = rmat24
    grp, gci = G.export_transpose()
    np.testing.assert_array_equal(grp.numpy(), tr[0])
    np.testing.assert_array_equal(gci.numpy(), tr[1])


def test_rmat24_pagerank_in_the_benchmark_configuration(T, rmat24):
    """Shared-memory blocks (B = 456 on GB300), fixed-point merge, 20 iterations: every rank
    against the oracle, mass 1, and bit-identical reruns."""
    g, G, rp, ci, tr = rmat24
    want = oracle.pagerank_pull(g.V, rp, ci, nthreads=CORES, transposed=tr)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem")
    assert P.staged
    r1 = T.pagerank_pull(G, P, merge="fixed")
    r2 = T.pagerank_pull(G, P, merge="fixed")
    got = r1.cpu().numpy()
    assert l1_rel(got, want) <= TOL
    assert abs(float(np.sum(got, dtype=np.float64)) - 1.0) < 1e-4
    assert torch.equal(r1, r2)
    assert l1_rel(T.pagerank_pull(G, None).cpu().numpy(), want) <= TOL


def test_rmat24_pagerank_renumbered_blocks(T, rmat24):
    """The benchmark's headline configuration: blocks cut after renumbering the vertices by
    out-degree (widest shared-memory blocks, gather tiles, merge ranges cut by pieces), fixed-point
    merge, 20 iterations: every rank against the oracle, mass 1, bit-identical reruns."""
    g, G, rp, ci, tr = rmat24
    want = oracle.pagerank_pull(g.V, rp, ci, nthreads=CORES, transposed=tr)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem", order="outdegree")
    assert P.staged and P.vertex_order == T.TC_ORDER_OUTDEGREE
    r1 = T.pagerank_pull(G, P)
    r2 = T.pagerank_pull(G, P)
    got = r1.cpu().numpy()
    assert l1_rel(got, want) <= TOL
    assert abs(float(np.sum(got, dtype=np.float64)) - 1.0) < 1e-4
    assert torch.equal(r1, r2)


def test_rmat24_bfs_bit_exact(T, rmat24):
    """Symmetrised R-MAT 24 (~521M directed edges), two seeded sources, direction-optimised with
    and without TOCAB pull levels, and pure pull (L2-rule blocks above the threshold, and 8
    blocks in every level)."""
    g = rmat24[0]
    gs = gg.symmetrize(g)
    Gs = T.graph_load_csr(gs.rowptr, gs.colidx, V=gs.V)
    Ps = T.tocab_partition(Gs, T.TC_PULL, 0, block_policy="l2")
    P8 = T.tocab_partition(Gs, T.TC_PULL, 8, smem_stage=-1)
    rp, ci = gs.numpy()
    for s in gg.sources(gs, 2, seed=13):
        want = oracle.bfs(gs.V, rp, ci, s)
        for thr, push in [(0.05, 1.0 / 24), (-1.0, 1.0 / 24), (0.05, 0.0)]:
            lv, st = T.bfs_pull(Gs, Ps, s, tocab_threshold=thr, push_threshold=push, return_stats=True)
            np.testing.assert_array_equal(lv.cpu().numpy(), want)
            assert st.reached == int((want >= 0).sum())
        # the benchmark's TOCAB configuration: 8 blocks, every pull level blocked
        lv, st = T.bfs_pull(Gs, P8, s, tocab_threshold=0.0, return_stats=True)
        np.testing.assert_array_equal(lv.cpu().numpy(), want)
        assert st.tocab_levels == st.levels


def test_rmat22_ppr_batch_sampled_columns(T):
    """256 sources on R-MAT 22 in one [V x 256] batch: four seeded columns against the oracle
    (columns are independent problems).  The last column's source is the vertex with the most
    in-edges, whose own row is the longest gather of every iteration."""
    g = gg.rmat(22, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    srcs = gg.sources(g, 256, seed=17)
    srcs[255] = int(torch.bincount(g.colidx.long(), minlength=g.V).argmax())
    R = T.ppr_batch(G, srcs, iters=20).cpu().numpy()
    cols = [0, 85, 170, 255]
    rp, ci = g.numpy()
    want = oracle.ppr_pull(g.V, rp, ci, [srcs[j] for j in cols], iters=20)
    for k, j in enumerate(cols):
        assert l1_rel(R[:, j], want[:, k]) <= TOL, j


def test_thousand_graphs_sampled(T):
    """1,000 R-MAT graphs (scales 10-16) in one persistent launch: 24 seeded graphs against the
    oracle one by one, and every graph's mass."""
    scales = gg.batch_scales(1000, 10, 16, seed=19)
    gb, off = gg.rmat_batch(scales, seed=19, device="cuda")
    M = T.multigraph_load(gb.rowptr, gb.colidx, off)
    r = T.pagerank_multi(M, iters=20).cpu().numpy()
    r_res = T.pagerank_multi(M, iters=20, lanes_per_vertex=T.TC_MULTI_RESIDENT).cpu().numpy()
    assert l1_rel(r_res, r) <= TOL  # the graph-per-CTA variant agrees with the grid-wide one
    rp, ci = gb.numpy()
    off = off.cpu().numpy().astype(np.int64)
    pick = np.random.default_rng(23).choice(len(off) - 1, size=24, replace=False)
    for k in pick:
        lo, hi = int(off[k]), int(off[k + 1])
        sub_rp = rp[lo:hi + 1] - rp[lo]
        sub_ci = ci[rp[lo]:rp[hi]] - lo
        want = oracle.pagerank_pull(hi - lo, sub_rp, sub_ci)
        assert l1_rel(r[lo:hi], want) <= TOL, k
    sums = np.add.reduceat(r.astype(np.float64), off[:-1])
    assert np.all(np.abs(sums - 1.0) < 1e-4)


def test_grid4096_bfs_bit_exact(T):
    """The 4096 x 4096 grid with 5% of its edges removed (about 8,000 levels of small frontiers):
    two seeded sources, direction-optimised with and without TOCAB pull levels, bit-exact."""
    g = gg.grid2d(4096, 4096, drop=0.05, seed=11, device="cuda")
    G = T.graph_load_csr(g.rowptr, g.colidx, V=g.V)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="l2")
    rp, ci = g.numpy()
    for s in gg.sources(g, 2, seed=13):
        want = oracle.bfs(g.V, rp, ci, s)
        for thr in (0.05, -1.0):
            lv, st = T.bfs_pull(G, P, s, tocab_threshold=thr, push_threshold=1.0 / 24, return_stats=True)
            np.testing.assert_array_equal(lv.cpu().numpy(), want)
            assert st.reached == int((want >= 0).sum())
            assert st.levels == int(want.max()) + 1
            assert st.resident_levels > st.levels // 2  # the small levels ran inside cluster launches


def test_rmat22_spmv_both_forms(T):
    """The SpMV row's workload (R-MAT 22, seeded values): the lane-group form and GC-pull with
    8 column blocks, every row against the FP64 oracle within the FP32 summation bound (the
    pieces of a row add one rounding per block), and GC-pull repeating bit for bit."""
    g = gg.rmat_host(22)  # the same graph as gg.rmat(22), generated in C
    G = _load(T, g)
    rp, ci = g.numpy()
    vals = gg.edge_values(g)
    x = torch.from_numpy(np.random.default_rng(22).standard_normal(g.V).astype(np.float32))
    v64, x64 = vals.numpy().astype(np.float64), x.numpy().astype(np.float64)
    want = oracle.spmv(g.V, rp, ci, v64, x64)
    mag = oracle.spmv(g.V, rp, ci, np.abs(v64), np.abs(x64))
    deg = np.diff(rp.astype(np.int64))
    y = T.spmv(G, vals.cuda(), x.cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(y - want) <= (deg + 6) * 2.0 ** -24 * mag + 1e-30)
    P = T.tocab_partition(G, T.TC_PUSH, 8, merge_range=8192)
    T.part_set_values(P, vals.cuda())
    yg = T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yg - want) <= (deg + 6 + 8) * 2.0 ** -24 * mag + 1e-30)
    assert np.array_equal(yg, T.spmv_tocab(P, x.cuda()).cpu().numpy().astype(np.float64))


def test_rmat21_bc_blocked_levels_bit_identical(T):
    """The BC row's larger workload (symmetrised R-MAT 21, 4 sources): blocked pull levels give
    tc_bc's scores bit for bit, and both match the FP64 oracle."""
    g = gg.symmetrize(gg.rmat_host(21).to("cuda")).to("cpu")
    G = _load(T, g)
    srcs = gg.sources(g, 4, seed=13)
    a = T.bc(G, srcs).cpu()
    P = T.tocab_partition(G, T.TC_PULL, 16, merge_range=8192, smem_stage=-1)
    b = T.bc(G, srcs, part=P).cpu()
    assert torch.equal(a, b)
    rp, ci = g.numpy()
    np.testing.assert_allclose(a.numpy(), oracle.bc(g.V, rp, ci, srcs), rtol=1e-11, atol=1e-8)
