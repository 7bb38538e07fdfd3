"""The seeded input generators shared by the oracle and the CUDA path (no method arithmetic):
determinism, and the structural promises every caller relies on (sorted, duplicate-free rows
without self loops; disjoint graphs in a batch; symmetric grids)."""
import numpy as np
import pytest
import torch

import graphgen as gg


def _check_csr(g):
    rp, ci = g.numpy()
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 0)
    assert ci.size == 0 or (ci.min() >= 0 and ci.max() < g.V)
    src = np.repeat(np.arange(g.V), np.diff(rp))
    assert not np.any(src == ci), "self loop"
    for v in range(min(g.V, 2000)):  # rows sorted and duplicate-free
        row = ci[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0)
    return rp, ci


@pytest.mark.parametrize("scale", [8, 12])
def test_rmat_is_deterministic_and_clean(scale):
    a, b = gg.rmat(scale), gg.rmat(scale)
    assert a.V == 1 << scale
    np.testing.assert_array_equal(a.rowptr.numpy(), b.rowptr.numpy())
    np.testing.assert_array_equal(a.colidx.numpy(), b.colidx.numpy())
    _check_csr(a)
    # edge factor 16 before dedup; R-MAT's skew makes duplicates common at small scales
    assert 0.5 * 16 * a.V < a.E <= 16 * a.V


def test_rmat_seed_changes_the_graph():
    a, b = gg.rmat(10), gg.rmat(10, seed=99)
    assert not (a.E == b.E and np.array_equal(a.colidx.numpy(), b.colidx.numpy()))


def test_erdos_renyi_and_powerlaw_are_clean():
    g = gg.erdos_renyi(3000, 20000, seed=5)
    _check_csr(g)
    assert 19000 < g.E <= 20000
    _check_csr(gg.powerlaw_config(5000, 6, 2.2, seed=3))


def test_grid_is_symmetric_with_degree_at_most_four():
    g = gg.grid2d(37, 41)
    rp, ci = _check_csr(g)
    assert np.diff(rp).max() <= 4
    src = np.repeat(np.arange(g.V), np.diff(rp))
    fwd = set(zip(src.tolist(), ci.tolist()))
    assert all((d, s) in fwd for s, d in fwd)
    full = 2 * (37 * 40 + 36 * 41)  # both directions of every grid edge
    assert 0.9 * full < g.E < full  # 5% of the undirected edges removed


def test_symmetrize_adds_every_reverse_edge():
    g = gg.rmat(9)
    s = gg.symmetrize(g)
    rp, ci = _check_csr(s)
    src = np.repeat(np.arange(s.V), np.diff(rp))
    edges = set(zip(src.tolist(), ci.tolist()))
    grp, gci = g.numpy()
    gsrc = np.repeat(np.arange(g.V), np.diff(grp))
    for u, v in zip(gsrc.tolist(), gci.tolist()):
        assert (u, v) in edges and (v, u) in edges


def test_rmat_batch_keeps_graphs_disjoint():
    scales = [6, 9, 4, 10, 7]
    g, off = gg.rmat_batch(scales, seed=19)
    off = off.numpy()
    assert off[0] == 0 and off[-1] == g.V and list(np.diff(off)) == [1 << s for s in scales]
    rp, ci = _check_csr(g)
    gid = np.searchsorted(off, np.arange(g.V), side="right") - 1
    src = np.repeat(np.arange(g.V), np.diff(rp))
    assert np.all(gid[src] == gid[ci]), "an edge joins two graphs"
    assert gg.batch_scales(1000, 10, 16, seed=19) == gg.batch_scales(1000, 10, 16, seed=19)


def test_sources_are_deterministic_and_have_edges():
    g = gg.rmat(12)
    s1, s2 = gg.sources(g, 16, seed=13), gg.sources(g, 16, seed=13)
    assert s1 == s2 and len(s1) == 16 and len(set(s1)) > 1
    deg = np.diff(g.rowptr.numpy())
    assert all(deg[s] > 0 for s in s1)


@pytest.mark.parametrize("scale,kw", [(8, {}), (12, {}), (12, {"permute_seed": None}),
                                      (13, {"a": 0.6, "b": 0.15, "c": 0.15, "seed": 9}),
                                      (10, {"a": 0.25, "b": 0.25, "c": 0.25}), (10, {"edge_factor": 4})])
def test_host_rmat_is_the_same_graph(scale, kw):
    """The C generator (the reference arm's) gives rmat()'s CSR exactly, thresholds of 2^32 included."""
    h, g = gg.rmat_host(scale, **kw), gg.rmat(scale, **kw)
    assert torch.equal(h.rowptr, g.rowptr) and torch.equal(h.colidx, g.colidx)
