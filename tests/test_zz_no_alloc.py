"""The allocation-free PageRank entry point, called through the C ABI.

tc_pagerank_pull_noalloc serves callers that may not allocate device memory (a plug-in
under a framework whose allocator owns the device memory, or a service with a memory
budget fixed at start-up): its scratch is a static device array of fixed size.  Here it
must agree with the allocating entry point (tc_pagerank_pull, unblocked) within the
tolerance of the other PageRank tests, on two calls in a row (the second call runs on the
scratch the first one left behind), and reject a vertex count above its limit.

This file is collected last on purpose so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import graphgen as gg

pytestmark = pytest.mark.gpu
TOL = 1e-5
MAX_V = 1 << 20


def _l1(got, want):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    return np.abs(got - want).sum() / np.abs(want).sum()


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_02241_gb300 as T
    T.lib()
    return T


def _noalloc(lib, V, rp, ci, outdeg, out, iters=20, damping=0.85, dangling=0):
    return lib.tc_pagerank_pull_noalloc(V, rp.data_ptr(), ci.data_ptr(), outdeg.data_ptr(), C.c_float(damping),
                                        iters, dangling, out.data_ptr(), torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("graph", ["rmat14", "er_dangling"])
def test_noalloc_matches_allocating_entry_point_twice(T, graph):
    g = gg.rmat(14) if graph == "rmat14" else gg.erdos_renyi(20000, 50000, seed=9)
    lib = T.lib()
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda())
    want = T.pagerank_pull(G, None, damping=0.85, iters=20).cpu().numpy()
    rp, ci = G.export_transpose(device="cuda")
    outdeg = (g.rowptr[1:] - g.rowptr[:-1]).to(torch.int32).cuda()
    for call in range(2):
        out = torch.full((g.V,), -1.0, dtype=torch.float32, device="cuda")
        st = _noalloc(lib, g.V, rp, ci, outdeg, out)
        assert st == 0, lib.tc_last_error()
        torch.cuda.synchronize()
        assert _l1(out.cpu().numpy(), want) <= TOL, f"call {call}"


def test_noalloc_drop_mode_and_zero_iterations(T):
    g = gg.rmat(12)
    lib = T.lib()
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda())
    rp, ci = G.export_transpose(device="cuda")
    outdeg = (g.rowptr[1:] - g.rowptr[:-1]).to(torch.int32).cuda()
    for iters, mode in [(7, 1), (0, 0)]:
        want = T.pagerank_pull(G, None, iters=iters, dangling=mode).cpu().numpy()
        out = torch.empty(g.V, dtype=torch.float32, device="cuda")
        assert _noalloc(lib, g.V, rp, ci, outdeg, out, iters=iters, dangling=mode) == 0
        torch.cuda.synchronize()
        assert _l1(out.cpu().numpy(), want) <= TOL


def test_noalloc_rejects_too_many_vertices(T):
    lib = T.lib()
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = _noalloc(lib, MAX_V + 1, dummy, dummy, dummy, out)
    assert st == -6  # TC_ERR_UNSUPPORTED
    assert b"static scratch" in lib.tc_last_error()
    assert _noalloc(lib, 0, dummy, dummy, dummy, out) == -6
