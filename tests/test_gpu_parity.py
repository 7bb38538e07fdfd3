"""GPU parity: every CUDA path through the C ABI against the FP64 CPU oracle.

Integer work (transpose, partition, BFS levels) must match bit-exactly; FP32 PageRank
must be within an L1 relative error of 1e-5 of the FP64 oracle after 20 iterations."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.gpu_util import l1_rel

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_02241_gb300 as T
    T.lib()
    return T


def _graphs():
    return {
        "rmat12": gg.rmat(12),
        "rmat14_noperm": gg.rmat(14, permute_seed=None),
        "er": gg.erdos_renyi(3000, 20000, seed=5),
        "grid": gg.grid2d(37, 41),
        "star": gg.star(300),
        "two": gg.from_edge_list(2, [(0, 1)]),
        "isolated": gg.from_edge_list(7, [(0, 1), (1, 0), (5, 6)]),
        "single": gg.empty_graph(1),
        "plc": gg.powerlaw_config(5000, 6, 2.2, seed=3),
    }


GRAPHS = _graphs()


def _load(T, g, device=True):
    rp, ci = (g.rowptr.cuda(), g.colidx.cuda()) if device else (g.rowptr, g.colidx)
    return T.graph_load_csr(rp, ci, V=g.V)


# ------------------------------------------------------------------ a1: load + transpose

@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("device", [True, False])
def test_transpose_bit_exact(T, name, device):
    g = GRAPHS[name]
    G = _load(T, g, device)
    rp, ci = G.export_transpose()
    wrp, wci = oracle.transpose(g.V, *g.numpy())
    np.testing.assert_array_equal(rp.numpy(), wrp)
    np.testing.assert_array_equal(ci.numpy(), wci)
    deg = np.diff(g.numpy()[0])
    assert G.num_dangling == int((deg == 0).sum())
    assert G.max_out_degree == int(deg.max(initial=0))


def test_device_memory_cap_gives_oom_and_recovers(T):
    """Failure injection on the host: a memory cap far below what a load needs makes the
    allocation fail with TC_ERR_OOM (naming the cap); after the cap is lifted the same call
    works and the results are unchanged."""
    g = GRAPHS["rmat12"]
    rp, ci = g.rowptr.cuda(), g.colidx.cuda()
    T.set_device_memory_limit(1)  # returns the cached blocks, so that `held` is what is in use
    T.set_device_memory_limit(T.device_memory_held() + 4096)
    try:
        with pytest.raises(T.TocabError) as e:
            T.graph_load_csr(rp, ci, V=g.V)
        assert e.value.status == -3 and "memory cap" in str(e.value)
    finally:
        T.set_device_memory_limit(0)
    G = T.graph_load_csr(rp, ci, V=g.V)
    assert l1_rel(T.pagerank_pull(G, None).cpu().numpy(), _oracle_pr(g)) <= TOL


def test_invalid_csr_rejected(T):
    bad_rp = torch.tensor([0, 2, 1], dtype=torch.int32)
    ci = torch.tensor([1, 0], dtype=torch.int32)
    with pytest.raises(T.TocabError) as e:
        T.graph_load_csr(bad_rp, ci)
    assert e.value.status == -2
    with pytest.raises(T.TocabError) as e:
        T.graph_load_csr(torch.tensor([0, 1, 2], dtype=torch.int32), torch.tensor([1, 5], dtype=torch.int32))
    assert e.value.status == -2


# ------------------------------------------------------------------ a2: partition

@pytest.mark.parametrize("name", ["rmat12", "er", "grid", "star", "isolated", "plc"])
@pytest.mark.parametrize("B", [1, 2, 3, 4, 7, 64])
@pytest.mark.parametrize("direction", ["pull", "push"])
def test_partition_bit_exact(T, name, B, direction):
    g = GRAPHS[name]
    if B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL if direction == "pull" else T.TC_PUSH, B)
    got = P.export()
    rp, ci = g.numpy()
    base = oracle.transpose(g.V, rp, ci) if direction == "pull" else (rp, ci)
    want = oracle.partition(g.V, base[0], base[1], P.block_width)
    assert got["B"] == want["B"]
    for key in ("blk_rows", "blk_edges", "rowptr", "id_map", "colidx"):
        np.testing.assert_array_equal(np.asarray(got[key], np.int64), np.asarray(want[key], np.int64), err_msg=key)


def test_partition_auto_width_uses_l2(T):
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 0)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert P.block_width == min(g.V, l2 // 11)


# ------------------------------------------------------------------ a3-a6: pull PageRank

def _oracle_pr(g, **kw):
    rp, ci = g.numpy()
    return oracle.pagerank_pull(g.V, rp, ci, **kw)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("B", [None, 1, 3, 4, 64])
def test_pagerank_pull_parity(T, name, B):
    g = GRAPHS[name]
    if B is not None and B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B) if B is not None else None
    r, st = T.pagerank_pull(G, P, return_stats=True)
    want = _oracle_pr(g)
    assert l1_rel(r.cpu().numpy(), want) <= TOL
    assert abs(st.dangling_mass - want[np.diff(g.numpy()[0]) == 0].sum()) <= 1e-5


@pytest.mark.parametrize("B", [None, 4])
def test_pagerank_pull_drop_mode_and_damping(T, B):
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B) if B else None
    for d, mode in [(0.85, "drop"), (0.5, "redistribute"), (0.0, "redistribute"), (1.0, "redistribute")]:
        r = T.pagerank_pull(G, P, damping=d, dangling=mode)
        assert l1_rel(r.cpu().numpy(), _oracle_pr(g, damping=d, dangling=mode)) <= TOL, (d, mode)


@pytest.mark.parametrize("iters", [0, 1, 2, 7])
def test_pagerank_pull_iteration_counts_and_host_output(T, iters):
    g = GRAPHS["er"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 3)
    out = torch.empty(g.V, dtype=torch.float32)  # host output
    T.pagerank_pull(G, P, iters=iters, out=out)
    assert l1_rel(out.numpy(), _oracle_pr(g, iters=iters)) <= TOL


def test_pagerank_pull_init(T):
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    init = torch.rand(g.V, generator=torch.Generator().manual_seed(0), dtype=torch.float64)
    init = init / init.sum()
    r = T.pagerank_pull(G, None, iters=5, init=init.float().cuda())
    want = _oracle_pr(g, iters=5, init=init.float().double().numpy())
    assert l1_rel(r.cpu().numpy(), want) <= TOL


def test_closed_form_star_on_gpu(T):
    n, d = 300, 0.85
    G = _load(T, GRAPHS["star"])
    hstar = (1 + d * n) / ((n + 1) * (1 + d))
    h20 = hstar + (-d) ** 20 * (1.0 / (n + 1) - hstar)
    for P in (None, T.tocab_partition(G, T.TC_PULL, 4)):
        r = T.pagerank_pull(G, P).cpu().numpy()
        assert abs(r[0] - h20) / h20 < 1e-5
        assert np.allclose(r[1:], (1 - h20) / n, rtol=1e-5)


def test_pull_result_is_deterministic(T):
    g = GRAPHS["rmat14_noperm"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 4)
    a = T.pagerank_pull(G, P).cpu()
    b = T.pagerank_pull(G, P).cpu()
    assert torch.equal(a, b)
    a = T.pagerank_pull(G, None).cpu()
    b = T.pagerank_pull(G, None).cpu()
    assert torch.equal(a, b)


# ------------------------------------------------------------------ a7: push PageRank

@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("B", [None, 1, 4, 64])
@pytest.mark.parametrize("lb", [0, 32])
def test_pagerank_push_parity(T, name, B, lb):
    """Push with fixed-point sums (the default): the oracle's ranks, bit for bit on reruns and
    the same bits whether a thread per edge (lb = 0) or the TWC rows (lb > 0) scatter them."""
    g = GRAPHS[name]
    if B is not None and B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PUSH, B) if B is not None else None
    r = T.pagerank_push(G, P, lb_warp_min=lb)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_push(G, P, lb_warp_min=lb).cpu())
    assert torch.equal(r.cpu(), T.pagerank_push(G, P, lb_warp_min=1 << 30).cpu())


@pytest.mark.parametrize("name", ["rmat12", "plc", "er", "isolated"])
@pytest.mark.parametrize("lb", [0, 8])
def test_pagerank_push_float_atomics(T, name, lb):
    """The paper's FP32-atomic sums: within the bar (order-dependent rounding)."""
    g = GRAPHS[name]
    G = _load(T, g)
    for P in (None, T.tocab_partition(G, T.TC_PUSH, min(4, g.V))):
        r = T.pagerank_push(G, P, lb_warp_min=lb, sums="float")
        assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL


def test_pagerank_push_float_rejected_for_pull(T):
    G = _load(T, GRAPHS["rmat12"])
    with pytest.raises(T.TocabError):
        T.pagerank_pull(G, None, merge="float")


def test_partition_direction_mismatch_rejected(T):
    G = _load(T, GRAPHS["rmat12"])
    P = T.tocab_partition(G, T.TC_PULL, 2)
    with pytest.raises(T.TocabError) as e:
        T.pagerank_push(G, P)
    assert e.value.status == -1


# ------------------------------------------------------------------ a8: BFS

BFS_GRAPHS = {
    "rmat12_sym": gg.symmetrize(gg.rmat(12)),
    "rmat12_dir": gg.rmat(12),
    "grid": gg.grid2d(37, 41),
    "path": gg.path(200),
    "star": gg.star(300),
    "isolated": gg.from_edge_list(7, [(0, 1), (1, 0), (5, 6)]),
    "single": gg.empty_graph(1),
}


@pytest.mark.parametrize("name", list(BFS_GRAPHS))
@pytest.mark.parametrize("mode", ["unblocked", "tocab_always", "tocab_threshold"])
def test_bfs_bit_exact(T, name, mode):
    g = BFS_GRAPHS[name]
    G = _load(T, g)
    P = None if mode == "unblocked" else T.tocab_partition(G, T.TC_PULL, min(4, g.V))
    thr = {"unblocked": -1.0, "tocab_always": 0.0, "tocab_threshold": 0.05}[mode]
    rp, ci = g.numpy()
    for s in gg.sources(g, 3, seed=13) + [0, g.V - 1]:
        lv, st = T.bfs_pull(G, P, s, tocab_threshold=thr, return_stats=True)
        want = oracle.bfs(g.V, rp, ci, s)
        np.testing.assert_array_equal(lv.cpu().numpy(), want)
        assert st.reached == int((want >= 0).sum())
        deg = np.diff(rp)
        assert st.edges_reached == int(deg[want >= 0].sum())
        if mode == "tocab_always" and st.levels > 0:
            assert st.tocab_levels == st.levels


def test_bfs_bad_source(T):
    G = _load(T, BFS_GRAPHS["path"])
    with pytest.raises(T.TocabError):
        T.bfs_pull(G, None, 200)


# ------------------------------------------------------------------ staged (shared-memory) gather

@pytest.mark.parametrize("name,B", [("rmat12", 4), ("rmat14_noperm", 16), ("er", 40), ("grid", 7),
                                    ("star", 5), ("plc", 5)])
@pytest.mark.parametrize("stage", [1, -1])
def test_pagerank_pull_staged_vs_unstaged(T, name, B, stage):
    g = GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, smem_stage=stage)
    assert P.staged == (stage == 1)
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL


@pytest.mark.parametrize("B", [None, 3])
def test_pagerank_pull_l2_window_changes_no_bit(T, B):
    """The L2 access-policy window only changes what the cache keeps: the ranks are bitwise those
    without it, for the unblocked and the unstaged TOCAB gather."""
    g = GRAPHS["rmat14_noperm"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, smem_stage=-1) if B is not None else None
    plain = T.pagerank_pull(G, P).cpu()
    win = T.pagerank_pull(G, P, l2_window=True).cpu()
    assert torch.equal(plain, win)
    assert l1_rel(win.numpy(), _oracle_pr(g)) <= TOL
    again = T.pagerank_pull(G, P).cpu()  # the set-aside is back: a plain call still agrees
    assert torch.equal(plain, again)


def test_smem_block_policy(T):
    g = gg.rmat(16)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem")
    assert P.staged and P.block_width % 32 == 0 and P.num_blocks >= 2
    assert P.staged_edges >= P.num_edges
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    # staged path is deterministic too (fixed-point merge)
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P).cpu())


def test_staged_requirement_rejected_when_width_too_large(T):
    g = gg.rmat(17)  # one block of 131,072 sources / destinations fits neither staged form
    G = _load(T, g)
    for d in (T.TC_PULL, T.TC_PUSH):
        with pytest.raises(T.TocabError) as e:
            T.tocab_partition(G, d, 1, smem_stage=1)
        assert e.value.status == -6


# ------------------------------------------------------------------ a9: batched personalised PageRank

@pytest.mark.parametrize("name,n", [("rmat12", 256), ("rmat12", 5), ("er", 130), ("grid", 1), ("plc", 300),
                                    ("isolated", 3)])
def test_ppr_batch_parity(T, name, n):
    g = GRAPHS[name]
    G = _load(T, g)
    rng = np.random.default_rng(n)
    srcs = rng.integers(0, g.V, n).astype(np.int32)
    srcs[0] = srcs[-1]  # a repeated source
    deg = np.diff(g.numpy()[0])
    if (deg == 0).any():
        srcs[len(srcs) // 2] = int(np.nonzero(deg == 0)[0][0])  # a dangling source
    R = T.ppr_batch(G, srcs, iters=20).cpu().numpy()
    rp, ci = g.numpy()
    want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
    for j in range(n):
        assert l1_rel(R[:, j], want[:, j]) <= TOL, j
    np.testing.assert_allclose(R.sum(axis=0), 1.0, atol=1e-5)


def test_ppr_batch_zero_iters_and_host_output(T):
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    srcs = [3, 9, 3]
    out = torch.empty((g.V, 3), dtype=torch.float32)
    T.ppr_batch(G, srcs, iters=0, out=out)
    want = np.zeros((g.V, 3))
    want[3, 0] = want[9, 1] = want[3, 2] = 1
    np.testing.assert_array_equal(out.numpy(), want)
    T.ppr_batch(G, srcs, iters=3, out=out)
    rp, ci = g.numpy()
    np.testing.assert_allclose(out.numpy(), oracle.ppr_pull(g.V, rp, ci, srcs, iters=3), rtol=2e-5, atol=1e-7)


def test_ppr_batch_rejects_bad_sources(T):
    G = _load(T, GRAPHS["rmat12"])
    with pytest.raises(T.TocabError):
        T.ppr_batch(G, [0, G.V])
    with pytest.raises(T.TocabError):
        T.ppr_batch(G, list(range(1025)))


# ------------------------------------------------------------------ merge modes

@pytest.mark.parametrize("merge", ["fixed", "ordered"])
@pytest.mark.parametrize("policy", ["smem", "l2"])
def test_pagerank_pull_merge_modes(T, merge, policy):
    g = gg.rmat(14)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 0 if policy == "smem" else 3, block_policy=policy)
    r = T.pagerank_pull(G, P, merge=merge)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P, merge=merge).cpu())


def test_removed_float_merge_mode_is_rejected(T):
    import ctypes as C
    from paper_1904_02241_gb300 import _lib as L
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 4)
    out = torch.empty(g.V, dtype=torch.float32, device="cuda")
    pp = L.tc_pr_params(0.85, 20, 0, L.TC_MEM_DEVICE, None, 0, 2, 0, 0)  # merge_mode 2
    st = T.lib().tc_pagerank_pull(G.handle, P.handle, C.byref(pp), out.data_ptr(), None,
                                  torch.cuda.current_stream().cuda_stream)
    assert st == -1


def _dense_range_graph():
    """V = 65536 sources, each with 32 out-edges into the first 4096 vertices: with 512 blocks
    of 128 sources and a merge range of 4096, range 0 holds about 1.6 M (block, row) entries,
    far more than the merge's chunk-to-slice map covers."""
    V = 65536
    u = np.repeat(np.arange(V, dtype=np.int64), 32)
    t = np.tile(np.arange(32, dtype=np.int64), V)
    d = (u * 37 + t * 131) % 4096
    return gg.from_edge_list(V, np.stack([u, d], 1), name="dense_range")


@pytest.mark.parametrize("B", [512, 2048])
def test_pagerank_pull_merge_dense_range(T, B):
    """Hundreds of pieces per vertex.  B = 2048 (32 sources per block) takes the three-part
    fixed-point merge, which every partition with 1,024 or more blocks uses."""
    g = _dense_range_graph()
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, merge_range=4096)
    assert P.num_blocks == B
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P).cpu())


@pytest.mark.parametrize("name,B,stage", [("rmat14_noperm", 1024, 0), ("plc", 1250, 0), ("rmat12", 2048, 0),
                                          ("rmat14_noperm", 2048, -1)])
def test_pagerank_pull_three_part_merge(T, name, B, stage):
    """1,024 blocks or more: the merge splits each partial into three fixed-point parts.  Small
    graphs give narrow blocks (W = 2..16 sources), so these run the unstaged gather; the dense-range
    test above runs the staged one with 2,048 blocks."""
    g = GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, smem_stage=stage)
    assert P.num_blocks >= 1024
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P).cpu())
    for d, mode in [(0.85, "drop"), (0.5, "redistribute")]:
        r = T.pagerank_pull(G, P, damping=d, dangling=mode)
        assert l1_rel(r.cpu().numpy(), _oracle_pr(g, damping=d, dangling=mode)) <= TOL


# ------------------------------------------------------------------ a10: many graphs in one launch

def _multi_oracle(g, off, **kw):
    rp, ci = g.numpy()
    off = np.asarray(off)
    out = np.zeros(g.V)
    for k in range(len(off) - 1):
        lo, hi = int(off[k]), int(off[k + 1])
        sub_rp = rp[lo:hi + 1] - rp[lo]
        sub_ci = ci[rp[lo]:rp[hi]] - lo
        if hi > lo:
            out[lo:hi] = oracle.pagerank_pull(hi - lo, sub_rp, sub_ci, **kw)
    return out


@pytest.fixture(scope="module")
def batch():
    return gg.rmat_batch([6, 9, 4, 10, 7, 8, 5, 9, 11, 3], seed=19)


@pytest.mark.parametrize("lanes", [0, -1, 1, 4, 8, 32, 1024])
@pytest.mark.parametrize("use_graph", [True, False])
def test_pagerank_multi_parity(T, batch, lanes, use_graph):
    g, off = batch
    M = T.multigraph_load(g.rowptr.cuda(), g.colidx.cuda(), off)
    r = T.pagerank_multi(M, lanes_per_vertex=lanes, use_graph=use_graph).cpu().numpy()
    want = _multi_oracle(g, off)
    assert l1_rel(r, want) <= TOL
    for k in range(len(off) - 1):  # every graph's mass is 1 on its own
        assert abs(r[off[k]:off[k + 1]].sum() - 1.0) < 1e-4


@pytest.mark.parametrize("lanes", [0, 1024])
def test_pagerank_multi_modes_and_reuse(T, batch, lanes):
    g, off = batch
    M = T.multigraph_load(g.rowptr.cuda(), g.colidx.cuda(), off)
    for iters, mode, d in [(0, "redistribute", 0.85), (3, "drop", 0.85), (20, "redistribute", 0.5),
                           (20, "redistribute", 0.85)]:
        r = T.pagerank_multi(M, iters=iters, dangling=mode, damping=d, lanes_per_vertex=lanes).cpu().numpy()
        assert l1_rel(r, _multi_oracle(g, off, iters=iters, dangling=mode, damping=d)) <= TOL


def test_multi_autotune_picks_a_variant(T, batch):
    g, off = batch
    M = T.multigraph_load(g.rowptr.cuda(), g.colidx.cuda(), off)
    best, times = T.multi_autotune(M)
    assert best in (-1, 1, 4, 8, 32, T.TC_MULTI_RESIDENT) and times[best] == min(times.values())
    assert T.TC_MULTI_RESIDENT in times  # these graphs fit one CTA's shared memory
    r = T.pagerank_multi(M).cpu().numpy()  # uses the tuned variant
    assert l1_rel(r, _multi_oracle(g, off)) <= TOL


def test_multi_resident_rejects_graphs_too_large_for_one_cta(T):
    """A cycle of 70,000 vertices has 70,000 non-dangling vertices: 280 KB of contributions, more
    than one CTA's shared memory, so the resident variant is refused and the tuner skips it."""
    g = gg.cycle(70000)
    M = T.multigraph_load(g.rowptr.cuda(), g.colidx.cuda(), [0, 70000])
    with pytest.raises(T.TocabError) as e:
        T.pagerank_multi(M, lanes_per_vertex=T.TC_MULTI_RESIDENT)
    assert e.value.status == -6
    best, times = T.multi_autotune(M)
    assert T.TC_MULTI_RESIDENT not in times and best in (-1, 1, 4, 8, 32)
    r = T.pagerank_multi(M).cpu().numpy()
    assert np.allclose(r, 1.0 / 70000, rtol=1e-5)


def _union(graphs):
    """Disjoint union of CSR graphs, with the vertex offset table."""
    rps, cis, off, e0 = [np.zeros(1, dtype=np.int64)], [], [0], 0
    for h in graphs:
        rp, ci = h.numpy()
        rps.append(rp[1:].astype(np.int64) + e0)
        cis.append(ci.astype(np.int64) + off[-1])
        e0 += len(ci)
        off.append(off[-1] + h.V)
    rp = torch.from_numpy(np.concatenate(rps).astype(np.int32))
    ci = torch.from_numpy(np.concatenate(cis).astype(np.int32))
    return gg.CSRGraph(off[-1], rp, ci, "union"), off


def test_multi_resident_edge_cases(T):
    """The resident variant splits every graph's in-edges evenly over 32 warps, so rows cross
    warp ranges.  Here a hub row of 20,000 in-edges crosses all of them, graphs without edges
    give warps empty ranges, and single vertices give empty graphs.  The result must match the
    oracle and repeat bit for bit."""
    parts = [gg.empty_graph(5), gg.star(20000), gg.path(3000), gg.cycle(1), gg.complete(40),
             gg.rmat(9, seed=5), gg.empty_graph(1), gg.path(700, directed=True), gg.cycle(33)]
    g, off = _union(parts)
    M = T.multigraph_load(g.rowptr.cuda(), g.colidx.cuda(), off)
    for mode in ("redistribute", "drop"):
        r = T.pagerank_multi(M, iters=20, dangling=mode, lanes_per_vertex=T.TC_MULTI_RESIDENT)
        want = _multi_oracle(g, off, iters=20, dangling=mode)
        assert l1_rel(r.cpu().numpy(), want) <= TOL, mode
        again = T.pagerank_multi(M, iters=20, dangling=mode, lanes_per_vertex=T.TC_MULTI_RESIDENT)
        assert torch.equal(r.cpu(), again.cpu())


def test_multigraph_rejects_cross_edges(T):
    g = gg.from_edge_list(4, [(0, 1), (1, 2), (2, 3)])
    with pytest.raises(T.TocabError) as e:
        T.multigraph_load(g.rowptr, g.colidx, [0, 2, 4])
    assert e.value.status == -2


# ------------------------------------------------------------------ load-balancing variants

@pytest.mark.parametrize("lb", [1, 8, 32, 1 << 30])
@pytest.mark.parametrize("kind", ["pull_unblocked", "pull_tocab", "push_tocab", "push_unblocked"])
def test_load_balancing_variants(T, lb, kind):
    g = GRAPHS["rmat14_noperm"]
    G = _load(T, g)
    if kind == "pull_unblocked":
        r = T.pagerank_pull(G, None, lb_warp_min=lb)
    elif kind == "pull_tocab":
        r = T.pagerank_pull(G, T.tocab_partition(G, T.TC_PULL, 4, smem_stage=-1), lb_warp_min=lb)
    elif kind == "push_tocab":
        r = T.pagerank_push(G, T.tocab_partition(G, T.TC_PUSH, 4), lb_warp_min=lb)
    else:
        r = T.pagerank_push(G, None, lb_warp_min=lb)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL


def test_per_block_load_balancing(T):
    g = GRAPHS["rmat14_noperm"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 4, smem_stage=-1)
    P.set_lb([1, 1 << 30, 32, 8][:P.num_blocks])
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    with pytest.raises(T.TocabError):
        P.set_lb([0] * P.num_blocks)
    P.set_lb(None)
    Pp = T.tocab_partition(G, T.TC_PUSH, 4)
    Pp.set_lb([1 << 30, 1, 8, 32][:Pp.num_blocks])
    assert l1_rel(T.pagerank_push(G, Pp).cpu().numpy(), _oracle_pr(g)) <= TOL


@pytest.mark.parametrize("name", list(BFS_GRAPHS))
@pytest.mark.parametrize("push", [1.0, 0.05, 0.002])
@pytest.mark.parametrize("tocab", [True, False])
def test_bfs_direction_optimised_bit_exact(T, name, push, tocab):
    g = BFS_GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, min(4, g.V)) if tocab else None
    rp, ci = g.numpy()
    for s in gg.sources(g, 3, seed=29) + [0]:
        lv, st = T.bfs_pull(G, P, s, tocab_threshold=0.0 if tocab else -1.0, push_threshold=push,
                            return_stats=True)
        want = oracle.bfs(g.V, rp, ci, s)
        np.testing.assert_array_equal(lv.cpu().numpy(), want)
        assert st.reached == int((want >= 0).sum())


@pytest.mark.parametrize("name", list(BFS_GRAPHS))
@pytest.mark.parametrize("cap", [0, 1, 5, 64, -1])
def test_bfs_resident_push_levels_bit_exact(T, name, cap):
    """Consecutive push levels inside one cluster launch: the same levels for every cap on the
    frontier (0 = host-driven levels only).  Small caps make the launches stop and restart; with
    push_threshold 0.05 the R-MAT graphs switch to pull levels after resident ones, which rebuild
    the frontier bitmap from the queue."""
    g = BFS_GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, min(4, g.V))
    rp, ci = g.numpy()
    for s in gg.sources(g, 3, seed=31) + [0]:
        want = oracle.bfs(g.V, rp, ci, s)
        for push, thr in ((1.0, -1.0), (0.05, 0.0), (0.05, -1.0)):
            lv, st = T.bfs_pull(G, P, s, tocab_threshold=thr, push_threshold=push, resident_edges=cap,
                                return_stats=True)
            np.testing.assert_array_equal(lv.cpu().numpy(), want)
            assert st.reached == int((want >= 0).sum())
            assert st.levels == int(want.max()) + 1
            assert 0 <= st.resident_levels <= st.push_levels <= st.levels
            if cap == 0:
                assert st.resident_levels == 0
            if st.levels <= T.TC_BFS_TRACE:
                kinds = list(st.level_kind)[:st.levels]
                assert st.resident_levels == sum(k == 3 for k in kinds)


def test_bfs_resident_levels_engage(T):
    """On a grid the levels run resident until the remaining out-edges fall below 14 times the
    frontier's (the last levels alternate pull and host-driven push), and on the R-MAT graph a
    pull level follows resident ones (the frontier bitmap rebuilt from the queue)."""
    g = BFS_GRAPHS["grid"]
    G = _load(T, g)
    rp, ci = g.numpy()
    want = oracle.bfs(g.V, rp, ci, 0)
    lv, st = T.bfs_pull(G, None, 0, tocab_threshold=-1.0, push_threshold=1.0, return_stats=True)
    np.testing.assert_array_equal(lv.cpu().numpy(), want)
    assert st.resident_levels > st.levels // 2
    g = BFS_GRAPHS["rmat12_sym"]
    G = _load(T, g)
    rp, ci = g.numpy()
    switched = False
    for s in gg.sources(g, 8, seed=37):
        lv, st = T.bfs_pull(G, None, s, tocab_threshold=-1.0, push_threshold=0.05, return_stats=True)
        np.testing.assert_array_equal(lv.cpu().numpy(), oracle.bfs(g.V, rp, ci, s))
        kinds = list(st.level_kind)[:min(st.levels, T.TC_BFS_TRACE)]
        switched |= any(a == 3 and b == 0 for a, b in zip(kinds, kinds[1:]))
    assert switched
    with pytest.raises(T.TocabError):
        T.bfs_pull(G, None, 0, push_threshold=0.05, resident_edges=(1 << 20) + 1)
    lv = T.bfs_pull(G, None, 0, push_threshold=0.05, resident_edges=1 << 20)  # the largest cap
    np.testing.assert_array_equal(lv.cpu().numpy(), oracle.bfs(g.V, rp, ci, 0))


@pytest.mark.parametrize("name,n,B", [("rmat12", 256, 3), ("rmat12", 40, 1), ("er", 130, 7), ("plc", 64, 4),
                                      ("grid", 33, 2)])
def test_ppr_batch_tocab_parity(T, name, n, B):
    g = GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, merge_range=256)
    rng = np.random.default_rng(n + B)
    srcs = rng.integers(0, g.V, n).astype(np.int32)
    R = T.ppr_batch(G, srcs, iters=20, part=P).cpu().numpy()
    rp, ci = g.numpy()
    want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
    for j in range(n):
        assert l1_rel(R[:, j], want[:, j]) <= TOL, j
    assert np.array_equal(R, T.ppr_batch(G, srcs, iters=20, part=P).cpu().numpy())  # deterministic


@pytest.mark.parametrize("tocab", [False, True])
def test_ppr_batch_long_rows_are_split(T, tocab):
    """A hub with more in-edges than a piece (2048 for rows, 1024 for tiles) runs as pieces."""
    g = gg.star(6000)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 2, merge_range=256) if tocab else None
    srcs = np.array([0, 1, 77, 5999, 0], np.int32)
    R = T.ppr_batch(G, srcs, iters=20, part=P).cpu().numpy()
    rp, ci = g.numpy()
    want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
    for j in range(len(srcs)):
        assert l1_rel(R[:, j], want[:, j]) <= TOL, j


def test_ppr_batch_persistent_replay_and_autotune(T):
    """The persistent batch is captured once and replayed: a second call with other sources into
    the same output must give that batch's answer, and after the autotuner has picked the hot
    block and launch width the answer is unchanged bit for bit."""
    g = GRAPHS["plc"]
    G = _load(T, g)
    rp, ci = g.numpy()
    out = torch.empty((g.V, 40), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(3)
    a = rng.integers(0, g.V, 40).astype(np.int32)
    b = rng.integers(0, g.V, 40).astype(np.int32)
    for srcs in (a, b, a):
        R = T.ppr_batch(G, srcs, iters=20, out=out).cpu().numpy()
        want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
        for j in range(len(srcs)):
            assert l1_rel(R[:, j], want[:, j]) <= TOL, j
    first = T.ppr_batch(G, a, iters=20, out=out).cpu().clone()
    hot, tile, times = T.ppr_autotune(G, a)
    assert hot >= 0 and tile in (0, 32, 64, 128) and min(times.values()) > 0
    again = T.ppr_batch(G, a, iters=20, out=out).cpu()
    assert torch.equal(first, again)  # the schedule changes no result


@pytest.mark.parametrize("tile", [0, 128, 64, 32])
@pytest.mark.parametrize("name,n", [("rmat12", 256), ("plc", 70), ("er", 33), ("isolated", 5)])
def test_ppr_batch_every_schedule(T, tile, name, n):
    """Every tile width of the persistent batch (0: whole rows), with and without evict-last
    rows, gives the oracle's answer, and all schedules give bit-identical results (each row's sum
    has a fixed order whatever the tiling)."""
    g = GRAPHS[name]
    G = _load(T, g)
    rp, ci = g.numpy()
    rng = np.random.default_rng(n + tile)
    srcs = rng.integers(0, g.V, n).astype(np.int32)
    want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
    outs = []
    for hot in (0, g.V // 3):
        T.ppr_set_tuning(G, hot=hot, tile=tile)
        R = T.ppr_batch(G, srcs, iters=20).cpu().numpy()
        for j in range(n):
            assert l1_rel(R[:, j], want[:, j]) <= TOL, (hot, j)
        outs.append(R)
    assert np.array_equal(outs[0], outs[1])
    T.ppr_set_tuning(G)


def test_ppr_batch_schedules_agree_on_long_rows(T):
    """A hub whose in-edges are cut into pieces, under every tile width."""
    g = gg.star(6000)
    G = _load(T, g)
    rp, ci = g.numpy()
    srcs = np.array([0, 1, 77, 5999, 0], np.int32)
    want = oracle.ppr_pull(g.V, rp, ci, srcs, iters=20)
    for tile in (0, 128, 64, 32):
        T.ppr_set_tuning(G, hot=-1, tile=tile)
        R = T.ppr_batch(G, srcs, iters=20).cpu().numpy()
        for j in range(len(srcs)):
            assert l1_rel(R[:, j], want[:, j]) <= TOL, (tile, j)


def test_ppr_set_tuning_rejects(T):
    G = _load(T, GRAPHS["rmat12"])
    for hot, tile in ((-2, 0), (0, 48), (0, 256)):
        with pytest.raises(T.TocabError):
            T.ppr_set_tuning(G, hot=hot, tile=tile)


def test_pagerank_push_fixed_point_signed_init(T):
    """Caller ranks of either sign go through the fixed-point sums (two's complement)."""
    g = GRAPHS["rmat12"]
    G = _load(T, g)
    rng = np.random.default_rng(11)
    init = torch.tensor(rng.standard_normal(g.V) / g.V, dtype=torch.float32)
    rp, ci = g.numpy()
    want = oracle.pagerank_push(g.V, rp, ci, iters=3, init=init.double().numpy())
    for P in (None, T.tocab_partition(G, T.TC_PUSH, 4)):
        r = T.pagerank_push(G, P, iters=3, init=init.cuda()).cpu().numpy()
        assert np.abs(r - want).sum() <= 1e-5 * np.abs(want).sum()


@pytest.mark.parametrize("name", ["rmat12", "plc", "er", "star", "isolated"])
@pytest.mark.parametrize("sums", ["fixed", "float"])
def test_pagerank_push_staged(T, name, sums):
    """The shared-memory staged push (smem_stage = 1): the oracle's ranks; with fixed-point sums
    the same bits as the global scatters."""
    g = GRAPHS[name]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PUSH, min(4, g.V), smem_stage=1)
    r = T.pagerank_push(G, P, sums=sums)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    if sums == "fixed":
        assert torch.equal(r.cpu(), T.pagerank_push(G, P, lb_warp_min=8).cpu())
        assert torch.equal(r.cpu(), T.pagerank_push(G, None).cpu())


