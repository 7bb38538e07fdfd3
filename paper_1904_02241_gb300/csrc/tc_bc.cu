// Betweenness centrality (the traversal benchmark of Sec. 3.3 and Sec. 4).
//
// Forward sweep: the shortest-path calculation of Alg. 3 (depth delta and shortest-path count
// sigma from one source), level by level, in the direction each level is cheaper in (Sec. 3.3's
// push-pull-push pattern: the first and last levels have small frontiers, the middle ones large):
//  * push: the frontier (the vertices of depth L, kept as a list) scatters over its out-edges;
//    an unreached target takes depth L+1 by compare-and-swap and every parent adds its sigma
//    with an FP64 atomic.  sigma counts paths, so every partial sum is an integer below 2^53
//    and exact: the result does not depend on the order of the additions.
//  * pull: every unreached vertex adds sigma over its in-neighbours of depth L (G^T), with no
//    atomics; a thread walks a short in-row, a warp a long one (in-degree >= 32, Sec. 3.2's
//    binning).  A vertex reads depth[u] of in-neighbours that other threads may set to L+1 in
//    the same launch; the old value (-1) and the new one both differ from L, so the read is
//    unaffected, and sigma[u] is read only for vertices of depth L, which no one writes now.
// Both directions append the vertices they reach to the next frontier list.
//
// Backward sweep: the dependency back-propagation of the BC the paper cites, over the level
// lists from the deepest, pulled over the out-edges of G: for a vertex v of depth L,
//   dep[v] = sum over out-neighbours w of depth L+1 of sigma[v] / sigma[w] * (1 + dep[w])
//          = sigma[v] * sum over those w of coef[w],   coef[w] = (1 + dep[w]) / sigma[w],
// so each vertex divides once (when its dependency is known) and each edge only adds; FP64
// division is slow on this GPU.  One warp per vertex: each lane adds its strided share of the
// row in order, then a fixed shuffle tree adds the lane sums; every vertex other than the source
// adds dep[v] to its score.  Operations are rounded one by one (no fused multiply-add).  A
// vertex's dependency reads only final values of the next level, so the order of a level's list
// (which the forward sweep fills as vertices are reached) does not change any result.
//
// sigma, the coefficients and the scores are FP64.
#include <vector>

#include "tc_common_dev.cuh"

namespace tc {

constexpr int BC_THREADS = 256;
constexpr int BC_WARPS = BC_THREADS / 32;
constexpr int BC_LONG = 32;  // rows with at least this many edges get a warp in pull levels

__global__ void k_bc_init(int32_t V, int32_t source, int32_t *depth, double *sigma, double *coef, int32_t *order) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        depth[v] = v == source ? 0 : -1;
        sigma[v] = v == source ? 1.0 : 0.0;
        coef[v] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) order[0] = source;  // level 0
}

__global__ void k_bc_zero(int32_t V, double *score) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        score[v] = 0.0;
}

// A vertex x joins level L+1: it is appended to the next frontier and its out-degree is added to
// the next frontier's out-edge count (the direction rule's m_f).
__device__ __forceinline__ void bc_reach(int32_t x, const int32_t *__restrict__ out_rowptr, int32_t *next,
                                         unsigned *next_count, unsigned long long *next_deg) {
    next[atomicAdd(next_count, 1u)] = x;
    atomicAdd(next_deg, (unsigned long long)(__ldg(out_rowptr + x + 1) - __ldg(out_rowptr + x)));
}

// out-degree of every frontier vertex (for the push level's edge prefix)
__global__ void k_bc_front_deg(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ front, int64_t nf,
                               int32_t *deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = front[i];
        deg[i] = __ldg(rowptr + u + 1) - __ldg(rowptr + u);
    }
}

// push level L, edge-balanced: thread t takes edges t, t + stride, ... of the frontier's
// concatenated out-rows (pre = exclusive prefix of their lengths, total = the sum) and finds its
// row by binary search, so a hub's row spreads over the whole grid.  The first edge to reach w
// claims it with a CAS on depth; every edge into a vertex of depth L+1 adds sigma[u] (integers
// below 2^53: exact in any order).
__global__ void __launch_bounds__(BC_THREADS) k_bc_push_edges(const int32_t *__restrict__ rowptr,
                                                              const int32_t *__restrict__ colidx,
                                                              const int32_t *__restrict__ front, int64_t nf,
                                                              const int64_t *__restrict__ pre, int64_t total,
                                                              int32_t L, int32_t *depth, double *sigma, int32_t *next,
                                                              unsigned *next_count, unsigned long long *next_deg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
        int64_t lo = 0, hi = nf;  // last i with pre[i] <= e
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(pre + mid) <= e) lo = mid; else hi = mid;
        }
        const int32_t u = __ldg(front + lo);
        const int32_t w = __ldg(colidx + __ldg(rowptr + u) + (e - __ldg(pre + lo)));
        int32_t dw = *(volatile int32_t *)(depth + w);
        if (dw == -1) {
            dw = atomicCAS(depth + w, -1, L + 1);
            if (dw == -1) {  // this edge reached w first
                dw = L + 1;
                bc_reach(w, rowptr, next, next_count, next_deg);
            }
        }
        if (dw == L + 1) atomicAdd(sigma + w, sigma[u]);
    }
}

// pull level L, short in-rows: a thread per unreached vertex
__global__ void __launch_bounds__(BC_THREADS) k_bc_pull(const int32_t *__restrict__ in_rowptr,
                                                        const int32_t *__restrict__ in_colidx,
                                                        const int32_t *__restrict__ out_rowptr, int32_t V, int32_t L,
                                                        int32_t *depth, double *sigma, int32_t *next,
                                                        unsigned *next_count, unsigned long long *next_deg) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        if (depth[v] != -1) continue;
        const int32_t s = in_rowptr[v], e = in_rowptr[v + 1];
        if (e - s >= BC_LONG) continue;  // k_bc_pull_long
        double acc = 0.0;
        bool hit = false;
        for (int32_t i = s; i < e; ++i) {
            const int32_t u = in_colidx[i];
            if (depth[u] == L) {
                acc = __dadd_rn(acc, sigma[u]);
                hit = true;
            }
        }
        if (hit) {
            depth[v] = L + 1;
            sigma[v] = acc;
            bc_reach((int32_t)v, out_rowptr, next, next_count, next_deg);
        }
    }
}

// pull level L, long in-rows: a warp per unreached vertex of the long-row list
__global__ void __launch_bounds__(BC_THREADS) k_bc_pull_long(const int32_t *__restrict__ in_rowptr,
                                                             const int32_t *__restrict__ in_colidx,
                                                             const int32_t *__restrict__ out_rowptr,
                                                             const int32_t *__restrict__ longrows, int32_t nlong,
                                                             int32_t L, int32_t *depth, double *sigma, int32_t *next,
                                                             unsigned *next_count, unsigned long long *next_deg) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * BC_WARPS;
    for (int64_t k = (blockIdx.x * (int64_t)BC_THREADS + threadIdx.x) >> 5; k < nlong; k += nw) {
        const int32_t v = longrows[k];
        if (depth[v] != -1) continue;  // the same value for the whole warp
        double acc = 0.0;
        bool hit = false;
        for (int32_t i = in_rowptr[v] + lane; i < in_rowptr[v + 1]; i += 32) {
            const int32_t u = in_colidx[i];
            if (depth[u] == L) {
                acc = __dadd_rn(acc, sigma[u]);
                hit = true;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, d));
        hit = __any_sync(0xffffffffu, hit);
        if (hit && lane == 0) {
            depth[v] = L + 1;
            sigma[v] = acc;
            bc_reach(v, out_rowptr, next, next_count, next_deg);
        }
    }
}

// Blocked pull level (TOCAB, Sec. 3.3 with sigma sums as the "next" values): local row r of a
// pull partition (block b's in-edges of destination id_map[r]) gets the sum of sigma over its
// sources of depth L, 0 when it has none or its destination is already reached.  A lane takes a
// row below 32 edges, a warp a longer one.  The sums are integers: exact in any order.
__global__ void __launch_bounds__(BC_THREADS) k_bc_block_level(const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const int32_t *__restrict__ id_map, int64_t R,
                                                               int32_t L, const int32_t *__restrict__ depth,
                                                               const double *__restrict__ sigma,
                                                               double *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * BC_WARPS;
    for (int64_t grp = (blockIdx.x * (int64_t)BC_THREADS + threadIdx.x) >> 5; grp * 32 < R; grp += nw) {
        const int64_t r = grp * 32 + lane;
        int32_t s = 0, e = 0;
        if (r < R && depth[__ldg(id_map + r)] == -1) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
        }
        double acc = 0.0;
        if (e - s < BC_LONG)
            for (int32_t i = s; i < e; ++i) {
                const int32_t u = __ldg(colidx + i);
                if (depth[u] == L) acc = __dadd_rn(acc, sigma[u]);
            }
        unsigned long_rows = __ballot_sync(0xffffffffu, e - s >= BC_LONG);
        while (long_rows) {
            const int l = __ffs(long_rows) - 1;
            long_rows &= long_rows - 1;
            const int32_t ls = __shfl_sync(0xffffffffu, s, l), le = __shfl_sync(0xffffffffu, e, l);
            double w = 0.0;
            for (int32_t i = ls + lane; i < le; i += 32) {
                const int32_t u = __ldg(colidx + i);
                if (depth[u] == L) w = __dadd_rn(w, sigma[u]);
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) w = __dadd_rn(w, __shfl_xor_sync(0xffffffffu, w, d));
            if (lane == l) acc = w;
        }
        if (r < R) partial[r] = acc;
    }
}

// The blocked level's merge (Fig. 5): CTA j adds the partial sums of vertices [j k, (j+1) k) over
// the blocks in order, then every unreached vertex with a nonzero sum takes depth L+1 and that
// sigma and joins the next frontier.
__global__ void __launch_bounds__(BC_THREADS) k_bc_block_merge(const double *__restrict__ partial,
                                                               const int32_t *__restrict__ id_map,
                                                               const int32_t *__restrict__ merge_off, int32_t B,
                                                               int32_t nranges, int32_t k, int32_t V, int32_t L,
                                                               const int32_t *__restrict__ out_rowptr,
                                                               int32_t *depth, double *sigma, int32_t *next,
                                                               unsigned *next_count, unsigned long long *next_deg) {
    extern __shared__ double bacc[];  // [k]
    for (int32_t j = blockIdx.x; j < nranges; j += gridDim.x) {
        const int32_t vbase = j * k;
        for (int32_t t = threadIdx.x; t < k; t += BC_THREADS) bacc[t] = 0.0;
        __syncthreads();
        for (int32_t b = 0; b < B; ++b) {
            const int32_t *o = merge_off + (int64_t)b * (nranges + 1) + j;
            const int32_t r0 = __ldg(o), r1 = __ldg(o + 1);
            for (int32_t r = r0 + threadIdx.x; r < r1; r += BC_THREADS) {
                const double x = partial[r];
                if (x != 0.0) bacc[__ldg(id_map + r) - vbase] = __dadd_rn(bacc[__ldg(id_map + r) - vbase], x);
            }
            __syncthreads();
        }
        for (int32_t t = threadIdx.x; t < k && vbase + t < V; t += BC_THREADS) {
            const double x = bacc[t];
            const int32_t v = vbase + t;
            if (x != 0.0 && depth[v] == -1) {
                depth[v] = L + 1;
                sigma[v] = x;
                bc_reach(v, out_rowptr, next, next_count, next_deg);
            }
        }
        __syncthreads();
    }
}

// dependency of v from t = the sum over its children of (1 + dep[w]) / sigma[w]: dep[v] =
// sigma[v] t goes to the score, and (1 + dep[v]) / sigma[v] to coef[v] for v's parents
__device__ __forceinline__ void bc_dep_update(int32_t v, double t, int32_t source, const double *__restrict__ sigma,
                                              double *coef, double *score) {
    const double sv = sigma[v];
    const double d = __dmul_rn(sv, t);
    coef[v] = __ddiv_rn(__dadd_rn(1.0, d), sv);  // for the parents of v, one level up
    if (v != source) score[v] = __dadd_rn(score[v], d);
}

// Dependencies of the vertices of depth L (those of depth L+1 are final), by out-degree class:
// up to BC_SMALL a group of 8 lanes (four vertices per warp), up to the hub degree a warp, above
// it a CTA (k_bc_backward_hub).  Each class adds in a fixed order, so scores repeat bit for bit.
constexpr int32_t BC_SMALL = 64;

__global__ void __launch_bounds__(BC_THREADS) k_bc_backward_small(const int32_t *__restrict__ rowptr,
                                                                  const int32_t *__restrict__ colidx,
                                                                  const int32_t *__restrict__ level_list, int64_t n,
                                                                  int32_t L, int32_t source, int32_t small_max,
                                                                  const int32_t *__restrict__ depth,
                                                                  const double *__restrict__ sigma, double *coef,
                                                                  double *score) {
    const int lane = threadIdx.x & 31, sub = lane & 7;
    const int64_t step = (int64_t)gridDim.x * BC_WARPS * 4;
    // warp-uniform loop: the shuffles below see the whole warp
    for (int64_t base = ((blockIdx.x * (int64_t)BC_THREADS + threadIdx.x) >> 5) * 4; base < n; base += step) {
        const int64_t k = base + (lane >> 3);
        int32_t v = -1, s = 0, e = 0;
        if (k < n) {
            v = level_list[k];
            s = rowptr[v];
            e = rowptr[v + 1];
            if (e - s > small_max) {  // a larger class
                v = -1;
                e = s;
            }
        }
        double t = 0.0;
        for (int32_t i = s + sub; i < e; i += 8) {
            const int32_t w = colidx[i];
            if (depth[w] == L + 1) t = __dadd_rn(t, coef[w]);
        }
#pragma unroll
        for (int q = 4; q > 0; q >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, q));
        if (sub == 0 && v >= 0) bc_dep_update(v, t, source, sigma, coef, score);
    }
}

__global__ void __launch_bounds__(BC_THREADS) k_bc_backward(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx,
                                                            const int32_t *__restrict__ level_list, int64_t n,
                                                            int32_t L, int32_t source, int32_t small_max,
                                                            int32_t hub_degree, const int32_t *__restrict__ depth,
                                                            const double *__restrict__ sigma, double *coef,
                                                            double *score) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * BC_WARPS;
    for (int64_t k = (blockIdx.x * (int64_t)BC_THREADS + threadIdx.x) >> 5; k < n; k += nw) {
        const int32_t v = level_list[k];
        const int32_t deg = rowptr[v + 1] - rowptr[v];
        if (deg <= small_max || deg > hub_degree) continue;  // the same for the whole warp
        double t = 0.0;  // sum of (1 + dep[w]) / sigma[w] over the children w
        for (int32_t e = rowptr[v] + lane; e < rowptr[v + 1]; e += 32) {
            const int32_t w = colidx[e];
            if (depth[w] == L + 1) t = __dadd_rn(t, coef[w]);
        }
#pragma unroll
        for (int q = 16; q > 0; q >>= 1) t = __dadd_rn(t, __shfl_xor_sync(0xffffffffu, t, q));
        if (lane == 0) bc_dep_update(v, t, source, sigma, coef, score);
    }
}

// the hubs of depth L: a CTA per hub of the graph's hub list, threads striding the out-row and a
// fixed-order block reduction (deterministic for the fixed launch shape); hubs at other depths
// leave at once
__global__ void __launch_bounds__(BC_THREADS) k_bc_backward_hub(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx,
                                                                const int32_t *__restrict__ hubs, int32_t L,
                                                                int32_t source, const int32_t *__restrict__ depth,
                                                                const double *__restrict__ sigma, double *coef,
                                                                double *score) {
    __shared__ double red[32];
    const int32_t v = hubs[blockIdx.x];
    if (depth[v] != L) return;  // the same for the whole CTA
    double t = 0.0;
    for (int32_t e = rowptr[v] + threadIdx.x; e < rowptr[v + 1]; e += BC_THREADS) {
        const int32_t w = colidx[e];
        if (depth[w] == L + 1) t = __dadd_rn(t, coef[w]);
    }
    t = block_sum<double>(t, red);
    if (threadIdx.x == 0) bc_dep_update(v, t, source, sigma, coef, score);
}

// A level runs in the push direction while its frontier's out-edges are fewer than
// 1 / BC_PUSH_RATIO of the out-edges of the vertices not yet reached (Beamer's rule).  The
// direction changes only the time: depths and the integer sigma sums are the same either way.
constexpr int64_t BC_PUSH_RATIO = 14;

struct BcScratch {
    DevBuf depth, sigma, coef, score, order, counter, longrows, bpartial;
    DevBuf fdeg, fpre, fws;  // push levels: frontier out-degrees, their prefix, scan scratch
    int32_t nlong = 0;
    std::vector<int64_t> off;  // level L of `order` is [off[L], off[L+1])
    int grid = 1;
    int setup(const tc_graph *g, bool need_score, cudaStream_t s, const tc_part *part = nullptr) {
        if (part) {
            TC_TRY(bpartial.alloc((size_t)(part->R > 0 ? part->R : 1) * 8));
            TC_CUDA(cudaFuncSetAttribute(k_bc_block_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)part->k * 8)));
        }
        const int32_t V = g->V;
        DeviceCaps caps;
        TC_TRY(device_caps(&caps));
        grid = caps.sms * 8;
        TC_TRY(depth.alloc((size_t)V * 4));
        TC_TRY(sigma.alloc((size_t)V * 8));
        TC_TRY(coef.alloc((size_t)V * 8));
        TC_TRY(order.alloc((size_t)V * 4));
        if (need_score) TC_TRY(score.alloc((size_t)V * 8));
        TC_TRY(counter.alloc(16));
        TC_TRY(fdeg.alloc((size_t)V * 4 + 16));
        TC_TRY(fpre.alloc((size_t)V * 8 + 16));
        TC_TRY(fws.alloc((size_t)(scan_ws_elems(V) + 16) * 8));
        TC_TRY(collect_hubs(g->in_rowptr.as<int32_t>(), V, BC_LONG - 1, &longrows, &nlong, s));
        return TC_OK;
    }
};

// Forward sweep from `source`: depth/sigma, and w.order holding the reached vertices level by
// level.  *max_depth = the deepest level (levels 0 .. *max_depth).  *pushed counts push levels.
static int bc_forward_impl(const tc_graph *g, const tc_part *part, int32_t source, BcScratch &w, cudaStream_t s,
                           int32_t *max_depth, int32_t *pushed) {
    const int32_t V = g->V;
    int32_t *depth = w.depth.as<int32_t>(), *order = w.order.as<int32_t>();
    double *sigma = w.sigma.as<double>();
    unsigned *cnt = w.counter.as<unsigned>();
    unsigned long long *ndeg = reinterpret_cast<unsigned long long *>(w.counter.as<char>() + 8);
    const int32_t *orp = g->out_rowptr.as<int32_t>();
    k_bc_init<<<w.grid, BC_THREADS, 0, s>>>(V, source, depth, sigma, w.coef.as<double>(), order);
    TC_LAUNCH_CHECK();
    w.off.assign(1, 0);
    w.off.push_back(1);
    // out-edges of the frontier (m_f) and of the vertices not yet reached (m_u)
    int32_t sdeg[2] = {0, 0};
    TC_CUDA(cudaMemcpyAsync(sdeg, orp + source, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    int64_t m_f = sdeg[1] - sdeg[0], m_u = g->E - m_f;
    int32_t L = 0, np = 0;
    for (;; ++L) {
        const int64_t f0 = w.off[(size_t)L], nf = w.off[(size_t)L + 1] - f0;
        const int64_t reached = w.off[(size_t)L + 1];
        TC_CUDA(cudaMemsetAsync(cnt, 0, 16, s));
        int32_t *next = order + reached;
        if (m_f * BC_PUSH_RATIO < m_u) {  // push, edge-balanced over the frontier's out-rows
            if (m_f > 0) {
                k_bc_front_deg<<<w.grid, BC_THREADS, 0, s>>>(orp, order + f0, nf, w.fdeg.as<int32_t>());
                TC_LAUNCH_CHECK();
                TC_TRY(scan_i32_to_i64_ws(w.fdeg.as<int32_t>(), nf, w.fpre.as<int64_t>(), w.fws.as<int64_t>(), s));
                const int64_t want = (m_f + BC_THREADS - 1) / BC_THREADS;
                const int grid = (int)(want < w.grid ? want : w.grid);
                k_bc_push_edges<<<grid, BC_THREADS, 0, s>>>(orp, g->out_colidx.as<int32_t>(), order + f0, nf,
                                                            w.fpre.as<int64_t>(), m_f, L, depth, sigma, next, cnt,
                                                            ndeg);
                TC_LAUNCH_CHECK();
            }
            ++np;
        } else if (part) {  // blocked pull level (TOCAB) and its merge
            if (part->R > 0) {
                k_bc_block_level<<<w.grid, BC_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                               part->id_map.as<int32_t>(), part->R, L, depth, sigma,
                                                               w.bpartial.as<double>());
                TC_LAUNCH_CHECK();
            }
            const size_t smem = (size_t)part->k * 8;
            const int mgrid = part->nranges < w.grid ? (part->nranges > 0 ? part->nranges : 1) : w.grid;
            k_bc_block_merge<<<mgrid, BC_THREADS, smem, s>>>(w.bpartial.as<double>(), part->id_map.as<int32_t>(),
                                                             part->merge_off.as<int32_t>(), part->B, part->nranges,
                                                             part->k, V, L, orp, depth, sigma, next, cnt, ndeg);
            TC_LAUNCH_CHECK();
        } else {
            k_bc_pull<<<w.grid, BC_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), orp, V,
                                                    L, depth, sigma, next, cnt, ndeg);
            TC_LAUNCH_CHECK();
            if (w.nlong > 0) {
                k_bc_pull_long<<<w.grid, BC_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(),
                                                             orp, w.longrows.as<int32_t>(), w.nlong, L, depth, sigma,
                                                             next, cnt, ndeg);
                TC_LAUNCH_CHECK();
            }
        }
        unsigned long long hc[2] = {0, 0};  // found (low word of the first), out-edges of the found
        TC_CUDA(cudaMemcpyAsync(hc, cnt, 16, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        const unsigned found = (unsigned)(hc[0] & 0xFFFFFFFFull);
        if (found == 0) break;
        w.off.push_back(reached + (int64_t)found);
        m_f = (int64_t)hc[1];
        m_u -= m_f;
    }
    *max_depth = L;
    if (pushed) *pushed = np;
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_bc_forward(const tc_graph *g, int32_t source, int out_mem, int32_t *depth_out, double *sigma_out,
                             void *stream) {
    using namespace tc;
    if (!g || !depth_out || !sigma_out) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: null graph or output");
    if (source < 0 || source >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: source outside [0, V)");
    if (out_mem != TC_MEM_HOST && out_mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: bad out_mem");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t V = g->V;
    BcScratch w;
    TC_TRY(w.setup(g, false, s));
    int32_t maxd = 0;
    TC_TRY(bc_forward_impl(g, nullptr, source, w, s, &maxd, nullptr));
    const cudaMemcpyKind kind = out_mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TC_CUDA(cudaMemcpyAsync(depth_out, w.depth.p, (size_t)V * 4, kind, s));
    TC_CUDA(cudaMemcpyAsync(sigma_out, w.sigma.p, (size_t)V * 8, kind, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

namespace tc {
static int bc_impl(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t num_sources, int out_mem,
                   double *scores_out, void *stream);
}  // namespace tc

extern "C" int tc_bc(const tc_graph *g, const int32_t *sources, int32_t num_sources, int out_mem, double *scores_out,
                     void *stream) {
    return tc::bc_impl(g, nullptr, sources, num_sources, out_mem, scores_out, stream);
}

extern "C" int tc_bc_tocab(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t num_sources,
                           int out_mem, double *scores_out, void *stream) {
    using namespace tc;
    if (!part) return fail(TC_ERR_INVALID_ARG, "tc_bc_tocab: null partition");
    if (part->g != g || part->dir != TC_PULL)
        return fail(TC_ERR_INVALID_ARG, "tc_bc_tocab: the partition must be a TC_PULL partition of this graph");
    if (part->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_bc_tocab: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if ((size_t)part->k * 8 > 200 * 1024)
        return fail(TC_ERR_UNSUPPORTED, "tc_bc_tocab: merge_range above 25,600");
    return bc_impl(g, part, sources, num_sources, out_mem, scores_out, stream);
}

namespace tc {
static int bc_impl(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t num_sources, int out_mem,
                   double *scores_out, void *stream) {
    if (!g || !scores_out || (num_sources > 0 && !sources))
        return fail(TC_ERR_INVALID_ARG, "tc_bc: null graph, sources or output");
    if (num_sources < 0) return fail(TC_ERR_INVALID_ARG, "tc_bc: num_sources < 0");
    if (out_mem != TC_MEM_HOST && out_mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "tc_bc: bad out_mem");
    for (int32_t k = 0; k < num_sources; ++k)
        if (sources[k] < 0 || sources[k] >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_bc: a source is outside [0, V)");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t V = g->V;
    if (V == 0) return TC_OK;
    BcScratch w;
    const bool dev_out = out_mem == TC_MEM_DEVICE;
    TC_TRY(w.setup(g, !dev_out, s, part));
    double *score = dev_out ? scores_out : w.score.as<double>();
    k_bc_zero<<<w.grid, BC_THREADS, 0, s>>>(V, score);
    TC_LAUNCH_CHECK();
    const int32_t small_max = BC_SMALL < g->hub_degree ? BC_SMALL : g->hub_degree;
    for (int32_t k = 0; k < num_sources; ++k) {
        int32_t maxd = 0;
        TC_TRY(bc_forward_impl(g, part, sources[k], w, s, &maxd, nullptr));
        for (int32_t L = maxd; L >= 0; --L) {
            const int64_t a = w.off[(size_t)L], n = w.off[(size_t)L + 1] - a;
            const int64_t want4 = (n + 4 * BC_WARPS - 1) / (4 * BC_WARPS);
            const int grid4 = (int)(want4 < w.grid ? (want4 > 0 ? want4 : 1) : w.grid);
            k_bc_backward_small<<<grid4, BC_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(),
                                                             w.order.as<int32_t>() + a, n, L, sources[k], small_max,
                                                             w.depth.as<int32_t>(), w.sigma.as<double>(),
                                                             w.coef.as<double>(), score);
            TC_LAUNCH_CHECK();
            const int64_t want = (n + BC_WARPS - 1) / BC_WARPS;
            const int grid = (int)(want < w.grid ? (want > 0 ? want : 1) : w.grid);
            k_bc_backward<<<grid, BC_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(),
                                                      w.order.as<int32_t>() + a, n, L, sources[k], small_max,
                                                      g->hub_degree,
                                                      w.depth.as<int32_t>(), w.sigma.as<double>(),
                                                      w.coef.as<double>(), score);
            TC_LAUNCH_CHECK();
            if (g->num_out_hubs > 0) {
                k_bc_backward_hub<<<g->num_out_hubs, BC_THREADS, 0, s>>>(
                    g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(), g->out_hubs.as<int32_t>(), L,
                    sources[k], w.depth.as<int32_t>(), w.sigma.as<double>(), w.coef.as<double>(), score);
                TC_LAUNCH_CHECK();
            }
        }
    }
    if (!dev_out) TC_CUDA(cudaMemcpyAsync(scores_out, score, (size_t)V * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}
}  // namespace tc
