"""FP64 CPU oracle for the TOCAB hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package.  The GPU library never calls it and shares no code with it.

Functions (each cites the paper passage it restates; see ``oracle.c``):
  transpose           -- G -> G^T (Sec. 2.1 CSR; Alg. 1 reads G^T)
  pagerank_pull       -- Alg. 1, Jacobi, FP64, dangling mass redistributed (or dropped)
  pagerank_push       -- Alg. 2, scatter form of the same iteration
  ppr_pull            -- personalised PageRank per source (teleport and dangling to s)
  bfs                 -- level-synchronous BFS hop levels (status arrays, Sec. 3.3)
  partition           -- TOCAB static 1D blocking with local IDs (Sec. 3.1, Fig. 3/4)
  bc_forward          -- Alg. 3: depth (delta) and shortest-path counts (sigma) from a source
  bc                  -- betweenness scores: Alg. 3 forward + dependency back-propagation
  spmv                -- y = A x for a CSR matrix with values (Sec. 4's SpMV benchmark)
  mlp_*               -- the cost model's MLP forward/backward in FP64 (oracle/mlp.py)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (OpenMP when the compiler supports it)."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            c = ctypes
            lib.orc_transpose.argtypes = [c.c_int32, c.c_int64, i32p, i32p, i32p, i32p]
            lib.orc_pagerank_pull.argtypes = [c.c_int32, i32p, i32p, i32p, c.c_double, c.c_int32,
                                              c.c_int32, c.c_void_p, f64p, c.c_int32]
            lib.orc_pagerank_push.argtypes = [c.c_int32, i32p, i32p, c.c_double, c.c_int32,
                                              c.c_int32, c.c_void_p, f64p]
            lib.orc_ppr_pull.argtypes = [c.c_int32, i32p, i32p, i32p, c.c_double, c.c_int32,
                                         c.c_int32, i32p, f64p]
            lib.orc_bfs.argtypes = [c.c_int32, i32p, i32p, c.c_int32, i32p]
            lib.orc_partition.argtypes = [c.c_int32, i32p, i32p, c.c_int32, c.c_int32,
                                          i64p, i64p, c.c_void_p, c.c_void_p, c.c_void_p]
            lib.orc_bc_forward.argtypes = [c.c_int32, i32p, i32p, c.c_int32, i32p, f64p, i32p,
                                           c.POINTER(c.c_int32)]
            lib.orc_bc.argtypes = [c.c_int32, i32p, i32p, c.c_int32, i32p, f64p]
            lib.orc_spmv.argtypes = [c.c_int32, i32p, i32p, f64p, f64p, f64p]
            for f in ("orc_transpose", "orc_pagerank_pull", "orc_pagerank_push", "orc_ppr_pull",
                      "orc_bfs", "orc_partition", "orc_bc_forward", "orc_bc", "orc_spmv"):
                getattr(lib, f).restype = c.c_int
            _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.int32)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def out_degree(rowptr) -> np.ndarray:
    rowptr = _i32(rowptr)
    return (rowptr[1:] - rowptr[:-1]).astype(np.int32)


def transpose(V: int, rowptr, colidx):
    """G (out-CSR) -> G^T (in-CSR), in-rows sorted by source."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    t_rowptr = np.zeros(V + 1, np.int32)
    t_colidx = np.zeros(max(colidx.size, 1), np.int32)
    _check(_load().orc_transpose(V, colidx.size, rowptr, colidx if colidx.size else np.zeros(1, np.int32),
                                 t_rowptr, t_colidx), "transpose")
    return t_rowptr, t_colidx[: colidx.size]


def pagerank_pull(V, rowptr, colidx, damping=0.85, iters=20, dangling="redistribute",
                  init=None, nthreads=1, transposed=None):
    """Alg. 1 in FP64 on G given as out-CSR (transposed internally unless given)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    t_rowptr, t_colidx = transposed if transposed is not None else transpose(V, rowptr, colidx)
    rank = np.zeros(V, np.float64)
    init_p = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.float64)
        init_p = init.ctypes.data
    tc = t_colidx if t_colidx.size else np.zeros(1, np.int32)
    _check(_load().orc_pagerank_pull(V, _i32(t_rowptr), tc, out_degree(rowptr), damping, iters,
                                     0 if dangling == "redistribute" else 1, init_p, rank,
                                     int(nthreads)), "pagerank_pull")
    return rank


def pagerank_push(V, rowptr, colidx, damping=0.85, iters=20, dangling="redistribute", init=None):
    """Alg. 2 in FP64 on G given as out-CSR."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    rank = np.zeros(V, np.float64)
    init_p = None
    if init is not None:
        init = np.ascontiguousarray(init, dtype=np.float64)
        init_p = init.ctypes.data
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    _check(_load().orc_pagerank_push(V, rowptr, cc, damping, iters,
                                     0 if dangling == "redistribute" else 1, init_p, rank),
           "pagerank_push")
    return rank


def ppr_pull(V, rowptr, colidx, sources, damping=0.85, iters=20, transposed=None):
    """Personalised PageRank per source; returns R[V, n] (row-major)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    t_rowptr, t_colidx = transposed if transposed is not None else transpose(V, rowptr, colidx)
    srcs = _i32(sources)
    R = np.zeros((V, srcs.size), np.float64)
    tc = t_colidx if t_colidx.size else np.zeros(1, np.int32)
    _check(_load().orc_ppr_pull(V, _i32(t_rowptr), tc, out_degree(rowptr), damping, iters,
                                srcs.size, srcs, R), "ppr_pull")
    return R


def bfs(V, rowptr, colidx, source):
    """Hop levels from ``source`` over out-edges; -1 = unreachable."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    lv = np.zeros(V, np.int32)
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    _check(_load().orc_bfs(V, rowptr, cc, int(source), lv), "bfs")
    return lv


def partition(V, rowptr, colidx, W: int):
    """TOCAB blocking of a CSR by column ranges of width W.

    Returns dict with blk_rows[B+1], blk_edges[B+1], rowptr[R+1] (int64 global edge
    offsets), id_map[R], colidx[E'] -- concatenated in block order."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    B = max(1, -(-V // W))
    blk_rows = np.zeros(B + 1, np.int64)
    blk_edges = np.zeros(B + 1, np.int64)
    lib = _load()
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    _check(lib.orc_partition(V, rowptr, cc, W, B, blk_rows, blk_edges, None, None, None), "partition")
    R, E = int(blk_rows[-1]), int(blk_edges[-1])
    rp = np.zeros(R + 1, np.int64)
    idm = np.zeros(max(R, 1), np.int32)
    col = np.zeros(max(E, 1), np.int32)
    _check(lib.orc_partition(V, rowptr, cc, W, B, blk_rows, blk_edges, rp.ctypes.data,
                             idm.ctypes.data, col.ctypes.data), "partition")
    return {"B": B, "W": W, "blk_rows": blk_rows, "blk_edges": blk_edges, "rowptr": rp,
            "id_map": idm[:R], "colidx": col[:E]}


def bc_forward(V, rowptr, colidx, source):
    """Alg. 3 from ``source`` over out-edges: (depth int32[V], -1 unreached; sigma float64[V])."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    depth = np.zeros(V, np.int32)
    sigma = np.zeros(V, np.float64)
    order = np.zeros(V, np.int32)
    count = ctypes.c_int32(0)
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    _check(_load().orc_bc_forward(V, rowptr, cc, int(source), depth, sigma, order, ctypes.byref(count)),
           "bc_forward")
    return depth, sigma


def bc(V, rowptr, colidx, sources=None):
    """Betweenness scores summed over ``sources`` (all vertices when None) and ordered targets."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    srcs = _i32(np.arange(V) if sources is None else sources)
    score = np.zeros(V, np.float64)
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    sp = srcs if srcs.size else np.zeros(1, np.int32)
    _check(_load().orc_bc(V, rowptr, cc, srcs.size, sp, score), "bc")
    return score


def spmv(nrows, rowptr, colidx, vals, x):
    """y = A x in FP64 for A in CSR (rows = outputs), values ``vals`` per stored entry."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(nrows, np.float64)
    cc = colidx if colidx.size else np.zeros(1, np.int32)
    vv = vals if vals.size else np.zeros(1, np.float64)
    xx = x if x.size else np.zeros(1, np.float64)
    _check(_load().orc_spmv(int(nrows), rowptr, cc, vv, xx, y), "spmv")
    return y


from .mlp import mlp_forward, mlp_backward, mlp_loss  # noqa: E402,F401
