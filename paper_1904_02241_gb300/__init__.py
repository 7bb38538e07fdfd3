"""GB300 (sm_103a) throughput-oriented cache blocking (TOCAB) for graph processing.

Thin Python binding over the C ABI of ``libtocab.so`` (declared in include/tocab.h).
Functions keep the C names without the ``tc_`` prefix:

  graph_load_csr(rowptr, colidx)            -> Graph     (tc_graph_load_csr)
  tocab_partition(graph, dir, num_blocks)   -> Partition (tc_tocab_partition)
  pagerank_pull(graph, part, ...)           -> ranks     (tc_pagerank_pull)
  pagerank_push(graph, part, ...)           -> ranks     (tc_pagerank_push)
  bfs_pull(graph, part, source, ...)        -> levels    (tc_bfs_pull)

Every step of the computation runs in the library's CUDA kernels; this module only
passes pointers, sizes and the current torch CUDA stream.  PyTorch provides device
memory and streams.  If the library is missing the import of a function fails loudly.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import (TC_BFS_TRACE, TC_DANGLING_DROP, TC_DANGLING_REDISTRIBUTE, TC_MEM_DEVICE,  # noqa: F401
                   TC_MEM_HOST, TC_MULTI_RESIDENT, TC_ORDER_NATURAL, TC_ORDER_OUTDEGREE, TC_PULL, TC_PUSH)

__all__ = ["graph_load_csr", "tocab_partition", "pagerank_pull", "pagerank_push", "bfs_pull", "ppr_batch", "ppr_autotune", "ppr_set_tuning", "part_set_values", "spmv_tocab",
           "multigraph_load",
           "pagerank_multi", "multi_autotune", "MultiGraph",
           "Graph", "Partition", "TocabError", "lib", "default_block_width", "set_device_memory_limit",
           "device_memory_held"]


class TocabError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = L.load()
        msg = lib.tc_last_error().decode(errors="replace")
        name = lib.tc_status_string(status).decode()
        super().__init__(f"{where}: {name} ({status}): {msg}")
        self.status = status


def lib():
    return L.load()


def set_device_memory_limit(nbytes: int) -> None:
    """tc_set_device_memory_limit: cap the library's device memory (0 removes the cap)."""
    _check(L.load().tc_set_device_memory_limit(int(nbytes)), "tc_set_device_memory_limit")


def device_memory_held() -> int:
    """tc_device_memory_held: bytes of device memory the library holds now."""
    return int(L.load().tc_device_memory_held())


def _check(status: int, where: str):
    if status != L.TC_OK:
        raise TocabError(status, where)


def _stream(stream=None) -> int:
    if stream is None:
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return 0
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _mem(t: torch.Tensor) -> int:
    return L.TC_MEM_DEVICE if t.is_cuda else L.TC_MEM_HOST


def _i32(t) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if t.dtype != torch.int32:
        raise TypeError(f"expected an int32 tensor, got {t.dtype}")
    return t.contiguous()


class Graph:
    """A graph resident on the current CUDA device (owns a tc_graph handle)."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle
        info = L.tc_graph_info()
        _check(L.load().tc_graph_get_info(self._h, C.byref(info)), "tc_graph_get_info")
        self.V = info.V
        self.E = info.E
        self.max_in_degree = info.max_in_degree
        self.max_out_degree = info.max_out_degree
        self.num_dangling = info.num_dangling

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            L.load().tc_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def export_transpose(self, device: str = "cpu"):
        rp = torch.empty(self.V + 1, dtype=torch.int32, device=device)
        ci = torch.empty(max(self.E, 1), dtype=torch.int32, device=device)
        _check(L.load().tc_graph_export_transpose(self._h, rp.data_ptr(), ci.data_ptr(), _mem(rp),
                                                  _stream()), "tc_graph_export_transpose")
        return rp, ci[: self.E]


class Partition:
    """A TOCAB partition of a Graph (owns a tc_part handle; keeps the graph alive)."""

    def __init__(self, handle: C.c_void_p, graph: Graph):
        self._h = handle
        self.graph = graph
        info = L.tc_part_info()
        _check(L.load().tc_part_get_info(self._h, C.byref(info)), "tc_part_get_info")
        self.dir = info.dir
        self.num_blocks = info.num_blocks
        self.block_width = info.block_width
        self.num_rows = info.num_rows
        self.num_edges = info.num_edges
        self.merge_range = info.merge_range
        self.num_hubs = info.num_hubs
        self.staged = bool(info.staged)
        self.staged_edges = info.staged_edges
        self.vertex_order = info.vertex_order
        self.num_ranges = info.num_ranges
        self.num_tiles = info.num_tiles
        self.num_sources = info.num_sources
        self.direct_blocks = info.direct_blocks
        self.num_direct = info.num_direct

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            L.load().tc_part_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_lb(self, warp_min_per_block=None):
        """tc_part_set_lb: per-subgraph load balancing (None clears the table)."""
        if warp_min_per_block is None:
            _check(L.load().tc_part_set_lb(self._h, None), "tc_part_set_lb")
            return
        t = torch.as_tensor(warp_min_per_block, dtype=torch.int32).contiguous().cpu()
        _check(L.load().tc_part_set_lb(self._h, t.data_ptr()), "tc_part_set_lb")

    def export(self):
        """Blocked CSR as host numpy arrays (blk_rows, blk_edges, rowptr, id_map, colidx)."""
        B, R, E = self.num_blocks, self.num_rows, self.num_edges
        br = torch.empty(B + 1, dtype=torch.int64)
        be = torch.empty(B + 1, dtype=torch.int64)
        rp = torch.empty(R + 1, dtype=torch.int32)
        im = torch.empty(max(R, 1), dtype=torch.int32)
        ci = torch.empty(max(E, 1), dtype=torch.int32)
        _check(L.load().tc_part_export(self._h, br.data_ptr(), be.data_ptr(), rp.data_ptr(), im.data_ptr(),
                                       ci.data_ptr(), L.TC_MEM_HOST, _stream()), "tc_part_export")
        return {"B": B, "W": self.block_width, "blk_rows": br.numpy(), "blk_edges": be.numpy(),
                "rowptr": rp.numpy(), "id_map": im.numpy()[:R], "colidx": ci.numpy()[:E]}

    def export_order(self):
        """tc_part_export_order: perm[n] = original ID of the vertex numbered n (numpy int32[V])."""
        perm = torch.empty(max(self.graph.V, 1), dtype=torch.int32)
        _check(L.load().tc_part_export_order(self._h, perm.data_ptr(), L.TC_MEM_HOST, _stream()),
               "tc_part_export_order")
        return perm.numpy()[: self.graph.V]


def graph_load_csr(rowptr, colidx, V: int | None = None, stream=None) -> Graph:
    """tc_graph_load_csr: out-edge CSR (int32 tensors on host or device) -> Graph."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    if V is None:
        V = rowptr.numel() - 1
    if rowptr.is_cuda != colidx.is_cuda and colidx.numel() > 0:
        raise ValueError("rowptr and colidx must live in the same memory space")
    h = C.c_void_p()
    ci_ptr = colidx.data_ptr() if colidx.numel() > 0 else None
    _check(L.load().tc_graph_load_csr(V, colidx.numel(), rowptr.data_ptr(), ci_ptr, _mem(rowptr),
                                      _stream(stream), C.byref(h)), "tc_graph_load_csr")
    return Graph(h)


def tocab_partition(graph: Graph, dir: int = L.TC_PULL, num_blocks: int = 0, l2_fraction: float = 0.0,
                    merge_range: int = 0, hub_degree: int = 0, block_policy: str = "l2", smem_stage: int = 0,
                    order: str = "natural", direct_blocks: int = 0, stream=None) -> Partition:
    """tc_tocab_partition: static 1D blocking.  num_blocks = 0 derives W from the L2 size
    (block_policy="l2", the paper's rule) or from one CTA's shared memory ("smem").
    order="outdegree" renumbers the vertices by out-degree before cutting the blocks (pull only);
    its single-edge pieces of the first direct_blocks blocks (0: none, -1: automatic) are direct."""
    policy = {"l2": L.TC_BLOCKS_L2, "smem": L.TC_BLOCKS_SMEM}[block_policy]
    vo = {"natural": L.TC_ORDER_NATURAL, "outdegree": L.TC_ORDER_OUTDEGREE}[order]
    pp = L.tc_part_params(l2_fraction, merge_range, hub_degree, policy, smem_stage, vo, direct_blocks)
    h = C.c_void_p()
    _check(L.load().tc_tocab_partition(graph.handle, dir, num_blocks, C.byref(pp), _stream(stream), C.byref(h)),
           "tc_tocab_partition")
    return Partition(h, graph)


def default_block_width(V: int, l2_bytes: int, l2_fraction: float = 0.0) -> int:
    return int(L.load().tc_default_block_width(V, l2_bytes, l2_fraction))


_MERGE = {"fixed": L.TC_MERGE_FIXED, "ordered": L.TC_MERGE_ORDERED, "float": L.TC_PUSH_FLOAT}


def _pagerank(fn, name, graph, part, damping, iters, dangling, out, init, profile, stream, merge="fixed",
              lb_warp_min=0, l2_window=False):
    if out is None:
        out = torch.empty(graph.V, dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or out.numel() < graph.V or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor with V elements")
    mode = {"redistribute": L.TC_DANGLING_REDISTRIBUTE, "drop": L.TC_DANGLING_DROP}[dangling] \
        if isinstance(dangling, str) else int(dangling)
    init_ptr = None
    if init is not None:
        if init.dtype != torch.float32 or init.is_cuda != out.is_cuda:
            raise ValueError("init must be float32 in the same memory space as out")
        init = init.contiguous()
        init_ptr = init.data_ptr()
    pp = L.tc_pr_params(float(damping), int(iters), mode, _mem(out), init_ptr, 1 if profile else 0,
                        _MERGE[merge], int(lb_warp_min), 1 if l2_window else 0)
    st = L.tc_pr_stats()
    _check(fn(graph.handle, part.handle if part is not None else None, C.byref(pp), out.data_ptr(),
              C.byref(st), _stream(stream)), name)
    return out, st


def pagerank_pull(graph: Graph, part: Partition | None = None, damping: float = 0.85, iters: int = 20,
                  dangling="redistribute", out: torch.Tensor | None = None, init: torch.Tensor | None = None,
                  profile: bool = False, stream=None, return_stats: bool = False, merge: str = "fixed",
                  lb_warp_min: int = 0, l2_window: bool = False):
    """tc_pagerank_pull (Alg. 1; TOCAB Alg. 4 + merge when part is given).
    merge: "fixed" (default) or "ordered" (both deterministic).
    l2_window: an L2 access-policy window over the contributions of the unstaged gathers."""
    r, st = _pagerank(L.load().tc_pagerank_pull, "tc_pagerank_pull", graph, part, damping, iters, dangling, out,
                      init, profile, stream, merge, lb_warp_min, l2_window)
    return (r, st) if return_stats else r


def pagerank_push(graph: Graph, part: Partition | None = None, damping: float = 0.85, iters: int = 20,
                  dangling="redistribute", out: torch.Tensor | None = None, init: torch.Tensor | None = None,
                  profile: bool = False, stream=None, return_stats: bool = False, lb_warp_min: int = 0,
                  sums: str = "fixed"):
    """tc_pagerank_push (Alg. 2; TOCAB Alg. 5 when part is given).  sums="fixed": 64-bit
    fixed-point reductions (bitwise repeatable); "float": FP32 atomics.  lb_warp_min = 0: a
    thread per edge; > 0: the thread/warp/CTA row mapping with that warp threshold."""
    r, st = _pagerank(L.load().tc_pagerank_push, "tc_pagerank_push", graph, part, damping, iters, dangling, out,
                      init, profile, stream, sums, lb_warp_min)
    return (r, st) if return_stats else r


def bc_forward(graph: Graph, source: int, stream=None):
    """tc_bc_forward (Alg. 3): (depth int32[V], -1 unreachable; sigma float64[V]) on the device."""
    depth = torch.empty(graph.V, dtype=torch.int32, device="cuda")
    sigma = torch.empty(graph.V, dtype=torch.float64, device="cuda")
    _check(L.load().tc_bc_forward(graph.handle, int(source), L.TC_MEM_DEVICE, depth.data_ptr(), sigma.data_ptr(),
                                  _stream(stream)), "tc_bc_forward")
    return depth, sigma


def bc(graph: Graph, sources=None, out: torch.Tensor | None = None, stream=None,
       part: "Partition | None" = None) -> torch.Tensor:
    """tc_bc: betweenness scores summed over ``sources`` (all vertices when None) -> float64[V].
    part: a TC_PULL partition of the graph for blocked pull levels (tc_bc_tocab; same result)."""
    src = torch.arange(graph.V, dtype=torch.int32) if sources is None else \
        torch.as_tensor(sources, dtype=torch.int32).reshape(-1).contiguous().cpu()
    if out is None:
        out = torch.empty(graph.V, dtype=torch.float64, device="cuda")
    if out.dtype != torch.float64 or out.numel() < graph.V or not out.is_contiguous():
        raise ValueError("out must be a contiguous float64 tensor with V elements")
    sp = src.data_ptr() if src.numel() else None
    if part is None:
        _check(L.load().tc_bc(graph.handle, sp, src.numel(), _mem(out), out.data_ptr(), _stream(stream)), "tc_bc")
    else:
        _check(L.load().tc_bc_tocab(graph.handle, part.handle, sp, src.numel(), _mem(out), out.data_ptr(),
                                    _stream(stream)), "tc_bc_tocab")
    return out


def spmv(matrix: Graph, vals: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None,
         stream=None) -> torch.Tensor:
    """tc_spmv: y = A x for the CSR loaded as ``matrix`` (rows = outputs); float32 on the device."""
    for t, n, what in ((vals, matrix.E, "vals"), (x, matrix.V, "x")):
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() < n:
            raise ValueError(f"{what} must be a contiguous float32 CUDA tensor with {n} elements")
    if out is None:
        out = torch.empty(matrix.V, dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < matrix.V:
        raise ValueError("out must be a contiguous float32 CUDA tensor with V elements")
    _check(L.load().tc_spmv(matrix.handle, vals.data_ptr() if vals.numel() else None, x.data_ptr(), out.data_ptr(),
                            L.TC_MEM_DEVICE, _stream(stream)), "tc_spmv")
    return out


def part_set_values(part: "Partition", vals: torch.Tensor, stream=None):
    """tc_part_set_values: the matrix values (CSR order, float32 on the device) for SpMV with
    TOCAB: GC-pull on a TC_PUSH partition, GC-push on a TC_PULL one."""
    if vals.dtype != torch.float32 or not vals.is_cuda or not vals.is_contiguous():
        raise ValueError("vals must be a contiguous float32 CUDA tensor")
    _check(L.load().tc_part_set_values(part.handle, vals.data_ptr() if vals.numel() else None, L.TC_MEM_DEVICE,
                                       _stream(stream)), "tc_part_set_values")


def spmv_tocab(part: "Partition", x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """tc_spmv_tocab: y = A x through a partition of A's graph: GC-pull for a TC_PUSH partition
    (fixed order), GC-push for a TC_PULL one (FP32 atomic adds)."""
    V = part.graph.V
    if x.dtype != torch.float32 or not x.is_cuda or not x.is_contiguous() or x.numel() < V:
        raise ValueError(f"x must be a contiguous float32 CUDA tensor with {V} elements")
    if out is None:
        out = torch.empty(V, dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or not out.is_cuda or not out.is_contiguous() or out.numel() < V:
        raise ValueError("out must be a contiguous float32 CUDA tensor with V elements")
    _check(L.load().tc_spmv_tocab(part.handle, x.data_ptr(), out.data_ptr(), L.TC_MEM_DEVICE, _stream(stream)),
           "tc_spmv_tocab")
    return out


def ppr_batch(graph: Graph, sources, damping: float = 0.85, iters: int = 20, out: torch.Tensor | None = None,
              profile: bool = False, stream=None, return_stats: bool = False, part: Partition | None = None):
    """tc_ppr_batch: personalised PageRank, one column per source -> [V, n] float32.
    part: a TC_PULL partition for the column-tiled TOCAB form (merge_range <= 256 advised)."""
    src = torch.as_tensor(sources, dtype=torch.int32).contiguous().cpu()
    n = src.numel()
    if out is None:
        out = torch.empty((graph.V, n), dtype=torch.float32, device="cuda")
    if out.dtype != torch.float32 or out.numel() < graph.V * n or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 tensor with V*n elements")
    pp = L.tc_pr_params(float(damping), int(iters), 0, _mem(out), None, 1 if profile else 0, 0, 0)
    st = L.tc_pr_stats()
    _check(L.load().tc_ppr_batch(graph.handle, part.handle if part is not None else None, src.data_ptr(), n,
                                 C.byref(pp), out.data_ptr(), C.byref(st), _stream(stream)), "tc_ppr_batch")
    return (out, st) if return_stats else out


def ppr_set_tuning(graph: Graph, hot: int = -1, tile: int = -1):
    """tc_ppr_set_tuning: the persistent batch's evict-last rows and tile width (0: whole rows;
    -1: default)."""
    _check(L.load().tc_ppr_set_tuning(graph.handle, int(hot), int(tile)), "tc_ppr_set_tuning")


def ppr_autotune(graph: Graph, sources, damping: float = 0.85, iters: int = 3, stream=None):
    """tc_ppr_autotune: time the persistent batch's tile widths and evict-last block sizes on these
    sources; returns (hot rows, tile width (0: whole rows), {(tile width, L2 fraction): ms}) and
    keeps the choice with the graph."""
    src = torch.as_tensor(sources, dtype=torch.int32).contiguous().cpu()
    pp = L.tc_pr_params(float(damping), int(iters), 0, L.TC_MEM_DEVICE, None, 0, 0, 0)
    hot = C.c_int32()
    tile = C.c_int32()
    times = (C.c_float * 16)()
    _check(L.load().tc_ppr_autotune(graph.handle, src.data_ptr(), src.numel(), C.byref(pp), C.byref(hot),
                                    C.byref(tile), times, _stream(stream)), "tc_ppr_autotune")
    keys = [(w, f) for w in (0, 128, 64, 32) for f in (0.0, 0.25, 0.5, 1.0)]
    return hot.value, tile.value, dict(zip(keys, list(times)))


class MultiGraph:
    """A batch of independent graphs on the current device (owns a tc_multigraph handle)."""

    def __init__(self, handle, V: int, E: int, n: int):
        self._h, self.V, self.E, self.num_graphs = handle, V, E, n
        self.tuned_lanes = 0

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            L.load().tc_multigraph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def multigraph_load(rowptr, colidx, vtx_off, stream=None) -> MultiGraph:
    """tc_multigraph_load: disjoint union CSR (global ids) + vertex offsets of its graphs."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    off = torch.as_tensor(vtx_off, dtype=torch.int32).contiguous().cpu()
    V = rowptr.numel() - 1
    h = C.c_void_p()
    ci_ptr = colidx.data_ptr() if colidx.numel() > 0 else None
    _check(L.load().tc_multigraph_load(off.numel() - 1, off.data_ptr(), V, colidx.numel(), rowptr.data_ptr(), ci_ptr,
                                       _mem(rowptr), _stream(stream), C.byref(h)), "tc_multigraph_load")
    return MultiGraph(h, V, colidx.numel(), off.numel() - 1)


def pagerank_multi(mg: MultiGraph, damping: float = 0.85, iters: int = 20, dangling="redistribute",
                   out: torch.Tensor | None = None, lanes_per_vertex: int = 0, ctas_per_sm: int = 0,
                   use_graph: bool = True, profile: bool = False, stream=None, return_stats: bool = False):
    """tc_pagerank_multi: PageRank on every graph of the batch in one persistent launch."""
    if out is None:
        out = torch.empty(mg.V, dtype=torch.float32, device="cuda")
    mode = {"redistribute": L.TC_DANGLING_REDISTRIBUTE, "drop": L.TC_DANGLING_DROP}[dangling]
    pp = L.tc_pr_params(float(damping), int(iters), mode, _mem(out), None, 1 if profile else 0, 0, 0)
    mp = L.tc_multi_params(int(lanes_per_vertex), int(ctas_per_sm), 1 if use_graph else 0)
    st = L.tc_pr_stats()
    _check(L.load().tc_pagerank_multi(mg.handle, C.byref(pp), C.byref(mp), out.data_ptr(), C.byref(st),
                                      _stream(stream)), "tc_pagerank_multi")
    return (out, st) if return_stats else out


def multi_autotune(mg: MultiGraph, damping: float = 0.85, iters: int = 20, stream=None):
    """tc_multi_autotune: time the lanes-per-vertex variants; returns (best, {lanes: ms})."""
    pp = L.tc_pr_params(float(damping), int(iters), 0, L.TC_MEM_DEVICE, None, 0, 0, 0)
    best = C.c_int32()
    times = (C.c_float * 6)()
    _check(L.load().tc_multi_autotune(mg.handle, C.byref(pp), C.byref(best), times, _stream(stream)),
           "tc_multi_autotune")
    mg.tuned_lanes = best.value
    # a negative time: the variant does not apply to this batch
    return best.value, {k: t for k, t in zip([-1, 1, 4, 8, 32, TC_MULTI_RESIDENT], list(times)) if t >= 0}


def bfs_pull(graph: Graph, part: Partition | None, source: int, tocab_threshold: float = 0.05,
             out: torch.Tensor | None = None, profile: bool = False, stream=None, return_stats: bool = False,
             push_threshold: float = 0.0, resident_edges: int = -1):
    """tc_bfs_pull: hop levels from source (-1 = unreachable).  push_threshold > 0 runs the
    small-frontier levels top-down (direction optimisation); consecutive push levels with at
    most resident_edges frontier vertices and out-edges run inside one cluster launch (0 = off,
    -1 = the library's default)."""
    if out is None:
        out = torch.empty(graph.V, dtype=torch.int32, device="cuda")
    if out.dtype != torch.int32 or out.numel() < graph.V or not out.is_contiguous():
        raise ValueError("out must be a contiguous int32 tensor with V elements")
    bp = L.tc_bfs_params(float(tocab_threshold), _mem(out), 1 if profile else 0, float(push_threshold),
                         int(resident_edges))
    st = L.tc_bfs_stats()
    _check(L.load().tc_bfs_pull(graph.handle, part.handle if part is not None else None, int(source), C.byref(bp),
                                out.data_ptr(), C.byref(st), _stream(stream)), "tc_bfs_pull")
    return (out, st) if return_stats else out
