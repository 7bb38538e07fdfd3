"""Seeded synthetic graph generators shared by the tests, the benchmark and the oracle side.

This module holds no PageRank, BFS or blocking arithmetic: it only draws graphs.
Every random decision comes from one counter-based hash of (seed, counter), computed
with 64-bit integer tensor arithmetic only, so the same call yields bit-identical
graphs on the CPU and on a CUDA device (``device=`` selects where the work runs).

Graph shapes follow the workloads of the paper's evaluation (Sec. 4, the benchmark
table): skewed power-law graphs (R-MAT, a Kronecker-style generator like Kron21),
graphs with no skew and poor locality (Erdos-Renyi), and graphs with a good layout
(a 2D grid, like the paper's Hollywood remark).  The paper's own datasets are not
available, so these seeded graphs stand in for them.

Output format everywhere: a directed graph G as an out-edge CSR,
``rowptr`` int32[V+1] and ``colidx`` int32[E], rows sorted by destination,
no self loops, no duplicate edges.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess

import numpy as np
import torch

MASK32 = 0xFFFFFFFF


@dataclasses.dataclass
class CSRGraph:
    """Out-edge CSR of a directed graph (int32 offsets and indices)."""
    V: int
    rowptr: torch.Tensor  # int32 [V+1]
    colidx: torch.Tensor  # int32 [E]
    name: str = ""

    @property
    def E(self) -> int:
        return int(self.colidx.numel())

    def to(self, device) -> "CSRGraph":
        return CSRGraph(self.V, self.rowptr.to(device), self.colidx.to(device), self.name)

    def numpy(self):
        return self.rowptr.cpu().numpy(), self.colidx.cpu().numpy()


# ----------------------------------------------------------------------------------------
# counter-based hash (Wellons' "lowbias32" integer hash, applied twice with the seed)
# ----------------------------------------------------------------------------------------

def _mul32(x: torch.Tensor, c: int) -> torch.Tensor:
    """(x * c) mod 2**32 for 0 <= x < 2**32 without int64 overflow."""
    hi = ((x >> 16) * c) & 0xFFFF
    lo = (x & 0xFFFF) * c
    return ((hi << 16) + lo) & MASK32


def _lowbias32(x: torch.Tensor) -> torch.Tensor:
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B)
    x = x ^ (x >> 16)
    return x


def hash_u32(seed: int, counter: torch.Tensor) -> torch.Tensor:
    """Uniform 32-bit value (held in int64) for each non-negative int64 counter."""
    s = int(seed) & MASK32
    k = int(_lowbias32(torch.tensor([s ^ 0x9E3779B9], dtype=torch.int64))[0])
    lo = counter & MASK32
    hi = (counter >> 32) & MASK32
    h = _lowbias32(lo ^ k)
    h = _lowbias32(h ^ ((hi + 0x68E31DA4 + s) & MASK32))
    return h


# ----------------------------------------------------------------------------------------
# edge lists -> CSR
# ----------------------------------------------------------------------------------------

def _csr_from_edges(V: int, src: torch.Tensor, dst: torch.Tensor, name: str) -> CSRGraph:
    """Drop self loops and duplicates; sort by (src, dst); build int32 CSR."""
    keep = src != dst
    key = src[keep] * V + dst[keep]
    key = torch.unique(key, sorted=True)
    s = key // V
    d = key - s * V
    counts = torch.bincount(s, minlength=V)
    rowptr = torch.zeros(V + 1, dtype=torch.int64, device=key.device)
    rowptr[1:] = torch.cumsum(counts, 0)
    assert int(rowptr[-1]) < 2**31, "int32 CSR limit"
    return CSRGraph(V, rowptr.to(torch.int32), d.to(torch.int32), name)


def from_edge_list(V: int, edges, name: str = "edges", device="cpu") -> CSRGraph:
    e = torch.as_tensor(np.asarray(edges, dtype=np.int64).reshape(-1, 2), device=device)
    return _csr_from_edges(V, e[:, 0].contiguous(), e[:, 1].contiguous(), name)


def _random_permutation(V: int, seed: int, device) -> torch.Tensor:
    v = torch.arange(V, dtype=torch.int64, device=device)
    key = (hash_u32(seed, v) << 31) | v  # unique keys, hash order
    return torch.argsort(key)


# ----------------------------------------------------------------------------------------
# workload generators
# ----------------------------------------------------------------------------------------

def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int | None = None, permute_seed: int | None = 7, device="cpu",
         chunk: int = 1 << 24) -> CSRGraph:
    """R-MAT graph: edge_factor * 2**scale draws, each edge descends ``scale`` quadrant levels.

    Quadrant probabilities (a, b, c, 1-a-b-c) are compared as 32-bit integer thresholds.
    Vertex IDs are then relabelled by a seeded random permutation (poor layout), self loops
    and duplicate edges are removed; the actual E is whatever remains.
    """
    V = 1 << scale
    M = edge_factor * V
    seed = 1 + scale if seed is None else seed
    ta = int(round(a * 2**32))
    tab = int(round((a + b) * 2**32))
    tabc = int(round((a + b + c) * 2**32))
    srcs, dsts = [], []
    for start in range(0, M, chunk):
        n = min(chunk, M - start)
        e = torch.arange(start, start + n, dtype=torch.int64, device=device)
        s = torch.zeros(n, dtype=torch.int64, device=device)
        d = torch.zeros(n, dtype=torch.int64, device=device)
        for lvl in range(scale):
            u = hash_u32(seed, e * scale + lvl)
            sbit = (u >= tab).to(torch.int64)
            dbit = ((u >= ta) & (u < tab)) | (u >= tabc)
            s = (s << 1) | sbit
            d = (d << 1) | dbit.to(torch.int64)
        srcs.append(s)
        dsts.append(d)
    src = torch.cat(srcs)
    dst = torch.cat(dsts)
    del srcs, dsts
    if permute_seed is not None:
        perm = _random_permutation(V, permute_seed, device)
        src = perm[src]
        dst = perm[dst]
    return _csr_from_edges(V, src, dst, f"rmat{scale}")


def erdos_renyi(V: int, M: int, seed: int = 3, device="cpu", chunk: int = 1 << 25) -> CSRGraph:
    """G(n, m)-style graph: M uniform (u, v) draws, self loops and duplicates dropped."""
    srcs, dsts = [], []
    for start in range(0, M, chunk):
        n = min(chunk, M - start)
        e = torch.arange(start, start + n, dtype=torch.int64, device=device)
        # uniform in [0, V) from a 32-bit draw: (u * V) >> 32 (V < 2**31)
        u1 = hash_u32(seed, 2 * e)
        u2 = hash_u32(seed, 2 * e + 1)
        srcs.append((u1 * V) >> 32)
        dsts.append((u2 * V) >> 32)
    return _csr_from_edges(V, torch.cat(srcs), torch.cat(dsts), f"er{V}")


def grid2d(rows: int, cols: int, drop: float = 0.05, seed: int = 11, device="cpu") -> CSRGraph:
    """4-neighbour 2D grid, both directions, row-major IDs; a seeded ``drop`` fraction of
    the undirected edges is removed (both directions of a removed edge go)."""
    V = rows * cols
    thr = int(round((1.0 - drop) * 2**32))
    r = torch.arange(rows, dtype=torch.int64, device=device)
    c = torch.arange(cols, dtype=torch.int64, device=device)
    # horizontal edges (r, c)-(r, c+1): ids 0 .. rows*(cols-1)-1
    hr, hc = torch.meshgrid(r, c[:-1], indexing="ij")
    hu = (hr * cols + hc).reshape(-1)
    hv = hu + 1
    # vertical edges (r, c)-(r+1, c)
    vr, vc = torch.meshgrid(r[:-1], c, indexing="ij")
    vu = (vr * cols + vc).reshape(-1)
    vv = vu + cols
    u = torch.cat([hu, vu])
    v = torch.cat([hv, vv])
    eid = torch.arange(u.numel(), dtype=torch.int64, device=device)
    keep = hash_u32(seed, eid) < thr
    u, v = u[keep], v[keep]
    return _csr_from_edges(V, torch.cat([u, v]), torch.cat([v, u]), f"grid{rows}x{cols}")


def symmetrize(g: CSRGraph) -> CSRGraph:
    """Add the reverse of every edge (then dedup)."""
    rowptr = g.rowptr.to(torch.int64)
    deg = rowptr[1:] - rowptr[:-1]
    src = torch.repeat_interleave(torch.arange(g.V, device=rowptr.device), deg)
    dst = g.colidx.to(torch.int64)
    return _csr_from_edges(g.V, torch.cat([src, dst]), torch.cat([dst, src]), g.name + "_sym")


def powerlaw_config(V: int, avg_deg: float, exponent: float, seed: int, device="cpu") -> CSRGraph:
    """Directed configuration-model-like graph: out-stub counts follow a discrete power law
    with the given exponent (mean scaled to ``avg_deg``), destinations drawn proportional to
    a second independent power-law weight.  Self loops and duplicates removed."""
    v = torch.arange(V, dtype=torch.int64, device=device)
    u = (hash_u32(seed, v).to(torch.float64) + 0.5) / 2**32
    w = (1.0 - u) ** (-1.0 / (exponent - 1.0))          # Pareto(x_min = 1)
    w = torch.clamp(w, max=float(V) ** 0.5 * 8)
    deg = torch.floor(w * (avg_deg / float(w.mean()))).to(torch.int64)
    M = int(deg.sum())
    src = torch.repeat_interleave(v, deg)
    # destination weights: second hash stream, inverse-CDF sample by searchsorted
    u2 = (hash_u32(seed + 7919, v).to(torch.float64) + 0.5) / 2**32
    w2 = (1.0 - u2) ** (-1.0 / (exponent - 1.0))
    cdf = torch.cumsum(w2, 0)
    cdf = cdf / cdf[-1]
    e = torch.arange(M, dtype=torch.int64, device=device)
    ue = (hash_u32(seed + 104729, e).to(torch.float64) + 0.5) / 2**32
    dst = torch.clamp(torch.searchsorted(cdf, ue), max=V - 1)
    return _csr_from_edges(V, src, dst, f"plc{V}")


# ----------------------------------------------------------------------------------------
# tiny graphs with closed-form answers
# ----------------------------------------------------------------------------------------

def cycle(n: int) -> CSRGraph:
    return from_edge_list(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def complete(n: int) -> CSRGraph:
    return from_edge_list(n, [(i, j) for i in range(n) for j in range(n) if i != j], f"K{n}")


def star(n: int) -> CSRGraph:
    """Hub 0 and leaves 1..n, edges in both directions."""
    e = [(0, i) for i in range(1, n + 1)] + [(i, 0) for i in range(1, n + 1)]
    return from_edge_list(n + 1, e, f"star{n}")


def path(n: int, directed: bool = False) -> CSRGraph:
    e = [(i, i + 1) for i in range(n - 1)]
    if not directed:
        e += [(i + 1, i) for i in range(n - 1)]
    return from_edge_list(n, e, f"path{n}")


def empty_graph(V: int) -> CSRGraph:
    return CSRGraph(V, torch.zeros(V + 1, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
                    f"empty{V}")


def random_small(V: int, M: int, seed: int) -> CSRGraph:
    """Small uniform random digraph (test sizes)."""
    return erdos_renyi(V, M, seed=seed)


def sources(g: CSRGraph, count: int, seed: int = 13, symmetric: bool = True) -> list[int]:
    """``count`` seeded BFS/PPR sources drawn uniformly among vertices with out-degree > 0."""
    rowptr = g.rowptr.cpu().to(torch.int64)
    cand = torch.nonzero(rowptr[1:] > rowptr[:-1]).reshape(-1)
    if cand.numel() == 0:
        return [0] * count
    idx = hash_u32(seed, torch.arange(count, dtype=torch.int64))
    return [int(cand[int(i) % cand.numel()]) for i in idx]


def rmat_batch(scales, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 19, permute_seed: int | None = 7, device="cpu"):
    """Many independent R-MAT graphs drawn in one vectorised pass (same recipe as ``rmat`` per
    graph: edge_factor * 2**s draws, quadrant descent, per-graph random relabelling, self loops
    and duplicates removed).  Returns (CSRGraph of the disjoint union, vtx_off int32[n+1]):
    graph g owns the vertices [vtx_off[g], vtx_off[g+1])."""
    sc = torch.as_tensor(list(scales), dtype=torch.int64, device=device)
    n = sc.numel()
    Vg = torch.pow(torch.full_like(sc, 2), sc)
    Mg = edge_factor * Vg
    vtx_off = torch.zeros(n + 1, dtype=torch.int64, device=device)
    vtx_off[1:] = torch.cumsum(Vg, 0)
    M = int(Mg.sum())
    V = int(vtx_off[-1])
    gid_e = torch.repeat_interleave(torch.arange(n, device=device), Mg)
    e = torch.arange(M, dtype=torch.int64, device=device)
    ta = int(round(a * 2**32))
    tab = int(round((a + b) * 2**32))
    tabc = int(round((a + b + c) * 2**32))
    s_e = sc[gid_e]
    src = torch.zeros(M, dtype=torch.int64, device=device)
    dst = torch.zeros(M, dtype=torch.int64, device=device)
    for lvl in range(int(sc.max()) if n else 0):
        act = s_e > lvl
        u = hash_u32(seed, e * 32 + lvl)
        sbit = (u >= tab).to(torch.int64)
        dbit = (((u >= ta) & (u < tab)) | (u >= tabc)).to(torch.int64)
        src = torch.where(act, (src << 1) | sbit, src)
        dst = torch.where(act, (dst << 1) | dbit, dst)
    base = vtx_off[:-1][gid_e]
    src = src + base
    dst = dst + base
    del gid_e, s_e, e
    if permute_seed is not None:
        v = torch.arange(V, dtype=torch.int64, device=device)
        gid_v = torch.repeat_interleave(torch.arange(n, device=device), Vg)
        key = (gid_v << 32) | hash_u32(permute_seed, v)
        order = torch.argsort(key)            # vertices grouped by graph, hash order inside
        new_id = torch.empty_like(order)
        new_id[order] = v                     # rank in that order = new global id
        src = new_id[src]
        dst = new_id[dst]
    g = _csr_from_edges(V, src, dst, f"rmat_batch{n}")
    return g, vtx_off.to(torch.int32)


def edge_values(g: CSRGraph, seed: int = 23, lo: float = -1.0, hi: float = 1.0) -> torch.Tensor:
    """Seeded FP32 value per stored entry (a weighted graph or a sparse matrix), uniform in
    [lo, hi), drawn from the counter hash of (seed, entry index): float32[E], on g's device."""
    e = torch.arange(g.E, dtype=torch.int64, device=g.colidx.device)
    u = (hash_u32(seed, e).to(torch.float64) + 0.5) / 2**32
    return (lo + (hi - lo) * u).to(torch.float32)


def batch_scales(count: int = 1000, lo: int = 10, hi: int = 16, seed: int = 19) -> list[int]:
    """Seeded scales drawn uniformly from [lo, hi] for a many-graph batch."""
    u = hash_u32(seed, torch.arange(count, dtype=torch.int64))
    return [lo + int(x) % (hi - lo + 1) for x in u]


# ----------------------------------------------------------------------------------------
# host R-MAT (C, OpenMP): the same graph as rmat(..., device="cpu"), generated in seconds
# instead of minutes at scale 24, for runs that must stay on the host
# ----------------------------------------------------------------------------------------

_HOST_DIR = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HOST_DIR, "_build", "libgg_host.so")
_host_lib = None


def build_native(force: bool = False) -> str:
    """Compile rmat_host.c with gcc (OpenMP when available) into graphgen/_build."""
    src = os.path.join(_HOST_DIR, "rmat_host.c")
    os.makedirs(os.path.dirname(_HOST_SO), exist_ok=True)
    if not force and os.path.exists(_HOST_SO) and os.path.getmtime(_HOST_SO) >= os.path.getmtime(src):
        return _HOST_SO
    tmp = _HOST_SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-fPIC", "-shared", "-std=c11", src, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _HOST_SO)
    return _HOST_SO


def rmat_host(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
              seed: int | None = None, permute_seed: int | None = 7) -> CSRGraph:
    """rmat() computed on the host cores by rmat_host.c: the identical CSR (same draws, same
    permutation, same deduplication and order), as CPU tensors."""
    global _host_lib
    if _host_lib is None:
        lib = ctypes.CDLL(build_native())
        lib.gg_rmat.restype = ctypes.c_int64
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
        lib.gg_free.argtypes = [ctypes.c_void_p]
        _host_lib = lib
    V = 1 << scale
    seed = 1 + scale if seed is None else seed
    ta = int(round(a * 2**32))
    tab = int(round((a + b) * 2**32))
    tabc = int(round((a + b + c) * 2**32))
    rowptr = np.zeros(V + 1, np.int64)
    ptr = ctypes.c_void_p()
    E = _host_lib.gg_rmat(scale, edge_factor, ta, tab, tabc, seed, -1 if permute_seed is None else permute_seed,
                          rowptr.ctypes.data, ctypes.byref(ptr))
    if E < 0:
        raise MemoryError("rmat_host: host allocation failed")
    try:
        col = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_int32)), (max(E, 1),))[:E].copy()
    finally:
        _host_lib.gg_free(ptr)
    assert E < 2**31, "int32 CSR limit"
    return CSRGraph(V, torch.from_numpy(rowptr.astype(np.int32)), torch.from_numpy(col), f"rmat{scale}")
