"""The allocation-free PageRank entry point, called through the C ABI.

tc_pagerank_pull_noalloc serves callers that may not allocate device memory (a plug-in
under a framework whose allocator owns the device memory, or a service with a memory
budget fixed at start-up): its scratch is a static device array of fixed size.  Here it
must agree with the allocating entry point (tc_pagerank_pull, unblocked) and with the FP64
oracle within the tolerance of the other PageRank tests, on two calls in a row (the second
call runs on the scratch the first one left behind), allocate nothing on calls after the
first, and reject a vertex count above its limit.

This file is collected last on purpose so that a run stopping at the first failure has
already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle

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


def _graph(name):
    return gg.rmat(14) if name == "rmat14" else gg.erdos_renyi(20000, 50000, seed=9)


@pytest.mark.parametrize("graph", ["rmat14", "er_dangling"])
def test_noalloc_matches_allocating_entry_point_twice(T, graph):
    g = _graph(graph)
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


@pytest.mark.parametrize("graph", ["rmat14", "er_dangling"])
def test_noalloc_matches_fp64_oracle(T, graph):
    """Directly against the FP64 oracle (Alg. 1 with dangling redistribution), not only
    against the other GPU path."""
    g = _graph(graph)
    lib = T.lib()
    oracle.build()
    rp_h, ci_h = g.numpy()
    want = oracle.pagerank_pull(g.V, rp_h, ci_h, damping=0.85, iters=20)
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda())
    rp, ci = G.export_transpose(device="cuda")
    outdeg = (g.rowptr[1:] - g.rowptr[:-1]).to(torch.int32).cuda()
    out = torch.empty(g.V, dtype=torch.float32, device="cuda")
    assert _noalloc(lib, g.V, rp, ci, outdeg, out) == 0, lib.tc_last_error()
    torch.cuda.synchronize()
    assert _l1(out.cpu().numpy(), want) <= TOL


def test_noalloc_allocates_nothing(T):
    """With the library's device-memory cap set to exactly what it holds, a further call must
    still succeed (any allocation would be refused), and neither the library's held bytes nor
    torch's allocated bytes may change across the call."""
    g = gg.rmat(12)
    lib = T.lib()
    G = T.graph_load_csr(g.rowptr.cuda(), g.colidx.cuda())
    rp, ci = G.export_transpose(device="cuda")
    outdeg = (g.rowptr[1:] - g.rowptr[:-1]).to(torch.int32).cuda()
    out = torch.empty(g.V, dtype=torch.float32, device="cuda")
    assert _noalloc(lib, g.V, rp, ci, outdeg, out) == 0  # first call on the device: module set-up
    torch.cuda.synchronize()
    T.set_device_memory_limit(max(T.device_memory_held(), 1))  # also returns cached blocks
    held = T.device_memory_held()
    torch_held = torch.cuda.memory_allocated()
    try:
        T.set_device_memory_limit(max(held, 1))
        for _ in range(2):
            assert _noalloc(lib, g.V, rp, ci, outdeg, out) == 0, lib.tc_last_error()
            torch.cuda.synchronize()
            assert T.device_memory_held() == held
            assert torch.cuda.memory_allocated() == torch_held
    finally:
        T.set_device_memory_limit(0)


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
