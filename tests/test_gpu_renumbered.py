"""Pull partitions renumbered by out-degree (TC_ORDER_OUTDEGREE) against the FP64 oracle.

The renumbering only changes which sources share a block (Sec. 3.1 cuts source ranges; here
the ranges are taken in a numbering by out-degree).  So the blocked CSR must equal the oracle's
blocking of the renumbered graph, bit for bit (the order of the sources inside one local row
is free), and PageRank must come back in the caller's numbering within the same 1e-5 L1 bar as
every other pull path, repeat bit for bit, and honour damping, dangling mode, iteration count,
initial ranks and host output."""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from tests.gpu_util import l1_rel

pytestmark = pytest.mark.gpu
TOL = 1e-5

GRAPHS = {
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


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_02241_gb300 as T
    T.lib()
    return T


def _load(T, g):
    return T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda(), V=g.V)


def _oracle_pr(g, **kw):
    rp, ci = g.numpy()
    return oracle.pagerank_pull(g.V, rp, ci, **kw)


def _want_order(g):
    """The numbering TC_ORDER_OUTDEGREE defines: vertices by out-degree, highest first, ties by
    ID, except that vertices without any edge come after those that have in-edges only."""
    rp, ci = g.numpy()
    deg = np.diff(rp.astype(np.int64))
    indeg = np.bincount(ci.astype(np.int64), minlength=g.V)
    isolated = ((deg == 0) & (indeg == 0)).astype(np.int64)
    return np.lexsort((np.arange(g.V), isolated, -deg)).astype(np.int32)


def _renumbered_transpose(g, perm):
    rp, ci = g.numpy()
    V = g.V
    inv = np.empty(V, np.int64)
    inv[perm] = np.arange(V)
    deg = np.diff(rp.astype(np.int64))
    src = np.repeat(np.arange(V, dtype=np.int64), deg)
    if src.size:
        g2 = gg.from_edge_list(V, np.stack([inv[src], inv[ci.astype(np.int64)]], 1))
        return oracle.transpose(V, *g2.numpy())
    return np.zeros(V + 1, np.int32), np.zeros(0, np.int32)


def _rows_sorted(rowptr, colidx):
    """(row, column) pairs of a blocked CSR in row order, columns ascending inside each row."""
    rowptr = np.asarray(rowptr, np.int64)
    rows = np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))
    cols = np.asarray(colidx, np.int64)
    o = np.lexsort((cols, rows))
    return rows[o], cols[o]


def _without_direct(want, Bd):
    """The oracle's blocking minus the single-edge local rows of blocks [0, Bd): the blocked CSR
    a partition with direct pieces keeps.  Returns it and the number of pieces taken out."""
    rp = np.asarray(want["rowptr"], np.int64)
    br = np.asarray(want["blk_rows"], np.int64)
    R = len(rp) - 1
    ln = np.diff(rp)
    drop = (ln == 1) & (np.arange(R) < br[min(Bd, len(br) - 1)])
    keep = ~drop
    edge_keep = np.repeat(keep, ln)
    new_ln = ln[keep]
    out = {"rowptr": np.concatenate([[0], np.cumsum(new_ln)]), "id_map": np.asarray(want["id_map"])[keep],
           "colidx": np.asarray(want["colidx"])[edge_keep]}
    kept_before = np.concatenate([[0], np.cumsum(keep)])
    out["blk_rows"] = kept_before[br]
    out["blk_edges"] = np.concatenate([[0], np.cumsum(new_ln)])[out["blk_rows"]]
    return out, int(drop.sum())


@pytest.mark.parametrize("name", ["rmat12", "er", "grid", "star", "isolated", "plc", "single", "two"])
@pytest.mark.parametrize("B", [1, 3, 4, 7, 64])
@pytest.mark.parametrize("direct", [0, -1, 2])
def test_renumbered_partition_matches_oracle_blocking(T, name, B, direct):
    """direct = 0: the oracle's blocking exactly; otherwise the same minus the single-edge
    pieces of the first direct_blocks blocks (-1: automatic), which are counted as direct."""
    g = GRAPHS[name]
    if B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, order="outdegree", direct_blocks=direct)
    assert P.vertex_order == T.TC_ORDER_OUTDEGREE
    perm = P.export_order()
    np.testing.assert_array_equal(perm, _want_order(g))
    deg = np.diff(g.numpy()[0])
    nz = int((deg > 0).sum())
    assert P.num_sources == nz
    W = P.block_width
    got = P.export()
    assert got["B"] == max(1, -(-nz // W))  # blocks past the last vertex with out-edges are dropped
    tr = _renumbered_transpose(g, perm)
    want = oracle.partition(g.V, tr[0], tr[1], W)
    Bg = got["B"]
    if direct == 0 or tr[1].size == 0:
        assert P.num_direct == 0
    else:
        if direct > 0:
            assert P.direct_blocks == min(direct, Bg)
        else:
            assert 1 <= P.direct_blocks <= Bg
        R_full = len(want["id_map"])
        want, nd = _without_direct(want, P.direct_blocks)
        assert P.num_direct == nd
        assert P.num_rows + nd == R_full
    np.testing.assert_array_equal(got["blk_rows"], want["blk_rows"][:Bg + 1])
    np.testing.assert_array_equal(got["blk_edges"], want["blk_edges"][:Bg + 1])
    assert (want["blk_rows"][Bg:] == want["blk_rows"][-1]).all()  # the oracle's extra blocks are empty
    np.testing.assert_array_equal(np.asarray(got["rowptr"], np.int64), want["rowptr"])
    np.testing.assert_array_equal(got["id_map"], want["id_map"])
    gr, gc = _rows_sorted(got["rowptr"], got["colidx"])
    wr, wc = _rows_sorted(want["rowptr"], want["colidx"])
    np.testing.assert_array_equal(gr, wr)
    np.testing.assert_array_equal(gc, wc)


def test_natural_partition_reports_identity_order(T):
    g = GRAPHS["rmat12"]
    P = T.tocab_partition(_load(T, g), T.TC_PULL, 4)
    assert P.vertex_order == T.TC_ORDER_NATURAL
    np.testing.assert_array_equal(P.export_order(), np.arange(g.V, dtype=np.int32))


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("B,stage", [(0, 0), (1, 0), (3, 0), (4, -1), (64, 0), (64, -1)])
def test_renumbered_pagerank_parity(T, name, B, stage):
    g = GRAPHS[name]
    if B > g.V:
        pytest.skip("B > V")
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, block_policy="smem", smem_stage=stage, order="outdegree")
    r, st = T.pagerank_pull(G, P, return_stats=True)
    want = _oracle_pr(g)
    assert l1_rel(r.cpu().numpy(), want) <= TOL
    assert abs(st.dangling_mass - want[np.diff(g.numpy()[0]) == 0].sum()) <= 1e-5
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P).cpu())  # deterministic


@pytest.mark.parametrize("B", [0, 4])
def test_renumbered_modes_iterations_init_and_host_output(T, B):
    g = GRAPHS["plc"]
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, block_policy="smem", order="outdegree")
    for d, mode in [(0.85, "drop"), (0.5, "redistribute"), (0.0, "redistribute"), (1.0, "redistribute")]:
        r = T.pagerank_pull(G, P, damping=d, dangling=mode)
        assert l1_rel(r.cpu().numpy(), _oracle_pr(g, damping=d, dangling=mode)) <= TOL, (d, mode)
    for iters in (0, 1, 2, 7):
        out = torch.empty(g.V, dtype=torch.float32)  # host output
        T.pagerank_pull(G, P, iters=iters, out=out)
        assert l1_rel(out.numpy(), _oracle_pr(g, iters=iters)) <= TOL, iters
    init = torch.rand(g.V, generator=torch.Generator().manual_seed(0), dtype=torch.float64)
    init = (init / init.sum()).float()
    for iters in (0, 5):
        r = T.pagerank_pull(G, P, iters=iters, init=init.cuda())
        want = _oracle_pr(g, iters=iters, init=init.double().numpy())
        assert l1_rel(r.cpu().numpy(), want) <= TOL, iters
    out = torch.empty(g.V, dtype=torch.float32)
    T.pagerank_pull(G, P, iters=5, init=init, out=out)  # host init and host output
    assert l1_rel(out.numpy(), _oracle_pr(g, iters=5, init=init.double().numpy())) <= TOL


@pytest.mark.parametrize("name", ["rmat12", "plc", "star", "isolated", "er"])
@pytest.mark.parametrize("direct", [0, 1, 3, -1])
@pytest.mark.parametrize("merge", ["fixed", "ordered"])
def test_renumbered_direct_pieces_parity(T, name, direct, merge):
    """Direct pieces (single-edge pieces of the first blocks, added by the merge from the
    contribution array) give the oracle's ranks in both merges, bit for bit on reruns, and agree
    with the partition without them (the other pieces' partial sums round differently: their
    rows fall on other chunk boundaries of the staged stream)."""
    g = GRAPHS[name]
    G = _load(T, g)
    B = min(8, g.V)
    P = T.tocab_partition(G, T.TC_PULL, B, block_policy="smem", order="outdegree", merge_range=256,
                          direct_blocks=direct)
    if direct != 0 and g.E > 0:
        assert P.num_direct > 0
    r = T.pagerank_pull(G, P, merge=merge)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P, merge=merge).cpu())
    if merge == "fixed":
        P0 = T.tocab_partition(G, T.TC_PULL, B, block_policy="smem", order="outdegree", merge_range=256,
                               direct_blocks=0)
        assert l1_rel(r.cpu().numpy(), T.pagerank_pull(G, P0, merge=merge).cpu().numpy()) <= TOL


@pytest.mark.parametrize("merge", ["fixed", "ordered"])
def test_renumbered_merge_modes(T, merge):
    g = gg.rmat(14)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem", order="outdegree", merge_range=1024)
    r = T.pagerank_pull(G, P, merge=merge)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P, merge=merge).cpu())


def test_renumbered_merge_ranges_balance_pieces(T):
    """R-MAT's hubs get few vertices per merge range, the tail many; no range exceeds the
    merge width, and the same ranks come out as with natural order."""
    g = gg.rmat(16)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem", order="outdegree", merge_range=2048)
    Pn = T.tocab_partition(G, T.TC_PULL, 0, block_policy="smem")
    assert P.num_rows < Pn.num_rows  # fewer (block, row) pieces: the point of the renumbering
    r = T.pagerank_pull(G, P).cpu().numpy()
    assert l1_rel(r, _oracle_pr(g)) <= TOL
    assert l1_rel(r, T.pagerank_pull(G, Pn).cpu().numpy()) <= 2 * TOL


def test_renumbered_partition_refused_where_unsupported(T):
    g = gg.symmetrize(GRAPHS["rmat12"])
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, 4, order="outdegree")
    with pytest.raises(T.TocabError) as e:
        T.bfs_pull(G, P, 0)
    assert e.value.status == -6
    with pytest.raises(T.TocabError) as e:
        T.ppr_batch(G, [0, 1], part=P)
    assert e.value.status == -6
    with pytest.raises(T.TocabError) as e:
        T.tocab_partition(G, T.TC_PUSH, 4, order="outdegree")
    assert e.value.status == -6
    with pytest.raises(T.TocabError) as e:
        T.tocab_partition(G, T.TC_PULL, 4, order="outdegree", merge_range=64)
    assert e.value.status == -1


@pytest.mark.parametrize("order", ["natural", "outdegree"])
@pytest.mark.parametrize("B", [1, 2])
def test_staged_gather_rows_longer_than_a_chunk(T, order, B):
    """Hub rows of 20,000 and 9,000 in-edges span many 512-edge warp chunks in which no row
    starts (the gather's fast path), cross warp and tile boundaries, and sit next to short rows."""
    hubs = [(u, 0) for u in range(1, 20001)] + [(u, 7) for u in range(3, 9003)]
    rest = [(0, u) for u in range(1, 20001, 3)] + [(u, u + 1) for u in range(1, 20000, 7)]
    g = gg.from_edge_list(20001, hubs + rest)
    G = _load(T, g)
    P = T.tocab_partition(G, T.TC_PULL, B, smem_stage=1, order=order)
    assert P.staged
    r = T.pagerank_pull(G, P)
    assert l1_rel(r.cpu().numpy(), _oracle_pr(g)) <= TOL
    assert torch.equal(r.cpu(), T.pagerank_pull(G, P).cpu())
