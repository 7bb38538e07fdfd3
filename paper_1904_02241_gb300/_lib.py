"""ctypes declarations of the C ABI in include/tocab.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtocab.so")

TC_OK = 0
TC_ERR_INVALID_ARG = -1
TC_ERR_INVALID_GRAPH = -2
TC_ERR_OOM = -3
TC_ERR_CUDA = -4
TC_ERR_TIMEOUT = -5
TC_ERR_UNSUPPORTED = -6
TC_MEM_HOST = 0
TC_MEM_DEVICE = 1
TC_PULL = 0
TC_PUSH = 1
TC_DANGLING_REDISTRIBUTE = 0
TC_DANGLING_DROP = 1


class tc_graph_info(C.Structure):
    _fields_ = [("V", C.c_int32), ("E", C.c_int64), ("max_in_degree", C.c_int32),
                ("max_out_degree", C.c_int32), ("num_dangling", C.c_int64), ("device", C.c_int32)]


TC_BLOCKS_L2 = 0
TC_BLOCKS_SMEM = 1


class tc_part_params(C.Structure):
    _fields_ = [("l2_fraction", C.c_float), ("merge_range", C.c_int32), ("hub_degree", C.c_int32),
                ("block_policy", C.c_int32), ("smem_stage", C.c_int32), ("vertex_order", C.c_int32),
                ("direct_blocks", C.c_int32)]


TC_ORDER_NATURAL = 0
TC_ORDER_OUTDEGREE = 1


class tc_part_info(C.Structure):
    _fields_ = [("dir", C.c_int32), ("num_blocks", C.c_int32), ("block_width", C.c_int32),
                ("num_rows", C.c_int64), ("num_edges", C.c_int64), ("merge_range", C.c_int32),
                ("num_hubs", C.c_int32), ("staged", C.c_int32), ("staged_edges", C.c_int64),
                ("vertex_order", C.c_int32), ("num_ranges", C.c_int32), ("num_tiles", C.c_int32),
                ("num_sources", C.c_int32), ("direct_blocks", C.c_int32), ("num_direct", C.c_int64)]


TC_MERGE_FIXED = 0
TC_MERGE_ORDERED = 1
TC_PUSH_FLOAT = 3
TC_MULTI_RESIDENT = 1024


class tc_pr_params(C.Structure):
    _fields_ = [("damping", C.c_float), ("iters", C.c_int32), ("dangling", C.c_int32),
                ("out_mem", C.c_int32), ("init", C.c_void_p), ("profile", C.c_int32),
                ("merge_mode", C.c_int32), ("lb_warp_min", C.c_int32), ("l2_window", C.c_int32)]


class tc_pr_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("launches", C.c_int32), ("ms_total", C.c_float),
                ("ms_gather", C.c_float), ("ms_merge", C.c_float), ("dangling_mass", C.c_double)]


class tc_multi_params(C.Structure):
    _fields_ = [("lanes_per_vertex", C.c_int32), ("ctas_per_sm", C.c_int32), ("use_graph", C.c_int32)]


class tc_bfs_params(C.Structure):
    _fields_ = [("tocab_threshold", C.c_float), ("out_mem", C.c_int32), ("profile", C.c_int32),
                ("push_threshold", C.c_float), ("resident_edges", C.c_int32)]


TC_BFS_TRACE = 64


class tc_bfs_stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("tocab_levels", C.c_int32), ("reached", C.c_int64),
                ("edges_reached", C.c_int64), ("ms_total", C.c_float), ("push_levels", C.c_int32),
                ("level_kind", C.c_int32 * TC_BFS_TRACE), ("level_frontier", C.c_int64 * TC_BFS_TRACE),
                ("level_ms", C.c_float * TC_BFS_TRACE), ("resident_levels", C.c_int32)]


VP = C.c_void_p
# name -> (restype, argtypes)
SIGNATURES = {
    "tc_status_string": (C.c_char_p, [C.c_int]),
    "tc_last_error": (C.c_char_p, []),
    "tc_version": (C.c_int, []),
    "tc_set_device_memory_limit": (C.c_int, [C.c_int64]),
    "tc_device_memory_held": (C.c_int64, []),
    "tc_graph_load_csr": (C.c_int, [C.c_int32, C.c_int64, VP, VP, C.c_int, VP, C.POINTER(VP)]),
    "tc_graph_free": (None, [VP]),
    "tc_graph_get_info": (C.c_int, [VP, C.POINTER(tc_graph_info)]),
    "tc_graph_export_transpose": (C.c_int, [VP, VP, VP, C.c_int, VP]),
    "tc_tocab_partition": (C.c_int, [VP, C.c_int, C.c_int32, C.POINTER(tc_part_params), VP, C.POINTER(VP)]),
    "tc_part_free": (None, [VP]),
    "tc_part_get_info": (C.c_int, [VP, C.POINTER(tc_part_info)]),
    "tc_part_export": (C.c_int, [VP, VP, VP, VP, VP, VP, C.c_int, VP]),
    "tc_part_export_order": (C.c_int, [VP, VP, C.c_int, VP]),
    "tc_part_set_lb": (C.c_int, [VP, VP]),
    "tc_default_block_width": (C.c_int32, [C.c_int32, C.c_int64, C.c_float]),
    "tc_pagerank_pull": (C.c_int, [VP, VP, C.POINTER(tc_pr_params), VP, C.POINTER(tc_pr_stats), VP]),
    "tc_pagerank_push": (C.c_int, [VP, VP, C.POINTER(tc_pr_params), VP, C.POINTER(tc_pr_stats), VP]),
    "tc_bfs_pull": (C.c_int, [VP, VP, C.c_int32, C.POINTER(tc_bfs_params), VP, C.POINTER(tc_bfs_stats), VP]),
    "tc_bc_forward": (C.c_int, [VP, C.c_int32, C.c_int, VP, VP, VP]),
    "tc_bc": (C.c_int, [VP, VP, C.c_int32, C.c_int, VP, VP]),
    "tc_bc_tocab": (C.c_int, [VP, VP, VP, C.c_int32, C.c_int, VP, VP]),
    "tc_spmv": (C.c_int, [VP, VP, VP, VP, C.c_int, VP]),
    "tc_part_set_values": (C.c_int, [VP, VP, C.c_int, VP]),
    "tc_spmv_tocab": (C.c_int, [VP, VP, VP, C.c_int, VP]),
    "tc_ppr_batch": (C.c_int, [VP, VP, VP, C.c_int32, C.POINTER(tc_pr_params), VP, C.POINTER(tc_pr_stats), VP]),
    "tc_ppr_autotune": (C.c_int, [VP, VP, C.c_int32, C.POINTER(tc_pr_params), C.POINTER(C.c_int32),
                                  C.POINTER(C.c_int32), VP, VP]),
    "tc_ppr_set_tuning": (C.c_int, [VP, C.c_int32, C.c_int32]),
    "tc_multigraph_load": (C.c_int, [C.c_int32, VP, C.c_int32, C.c_int64, VP, VP, C.c_int, VP, C.POINTER(VP)]),
    "tc_multigraph_free": (None, [VP]),
    "tc_pagerank_multi": (C.c_int, [VP, C.POINTER(tc_pr_params), C.POINTER(tc_multi_params), VP,
                                    C.POINTER(tc_pr_stats), VP]),
    "tc_multi_autotune": (C.c_int, [VP, C.POINTER(tc_pr_params), C.POINTER(C.c_int32), VP, VP]),
    "tc_graph_features": (C.c_int, [VP, VP]),
    "tc_part_features": (C.c_int, [VP, VP]),
    "tc_mlp_create": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, VP, C.POINTER(VP)]),
    "tc_mlp_free": (None, [VP]),
    "tc_mlp_num_params": (C.c_int64, [VP]),
    "tc_mlp_set_params": (C.c_int, [VP, VP]),
    "tc_mlp_get_params": (C.c_int, [VP, VP, VP]),
    "tc_mlp_forward": (C.c_int, [VP, VP, C.c_int32, VP, C.c_int, VP]),
    "tc_mlp_loss_grad": (C.c_int, [VP, VP, VP, C.c_int32, C.c_int, C.POINTER(C.c_double), VP]),
    "tc_mlp_adam_step": (C.c_int, [VP, C.c_float, C.c_float, C.c_float, C.c_float, VP]),
    "tc_mlp_train": (C.c_int, [VP, VP, VP, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_int,
                               C.POINTER(C.c_double), VP]),
    "tc_pagerank_pull_noalloc": (C.c_int, [C.c_int32, VP, VP, VP, C.c_float, C.c_int32, C.c_int32, VP, VP]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libtocab.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with "
                              "`python -m paper_1904_02241_gb300.build` (nvcc, sm_103a)")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
