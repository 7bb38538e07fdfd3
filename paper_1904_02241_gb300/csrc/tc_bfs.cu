// Topology-driven pull BFS with bitmap status arrays (Sec. 3.3, Fig. 1e/f).
//   unblocked level : warp per 32 vertices (one bitmap word); every unvisited vertex scans
//                     its in-edges with early exit until it finds a frontier source.
//   TOCAB level     : per block, a local "next" bit per local row (rows are scanned only
//                     over the block's sources), then a merge kernel ORs the local bits of
//                     all blocks per vertex range and writes levels, next and visited.
// Levels run TOCAB only when the frontier exceeds a fraction of V (Sec. 3.3).
#include <cooperative_groups.h>

#include "tc_common_dev.cuh"

namespace tc {

constexpr int BFS_THREADS = 256;
constexpr int BFS_WARPS = BFS_THREADS / 32;

__device__ __forceinline__ bool in_front(const uint32_t *__restrict__ front, int32_t u) {
    return (__ldg(front + (u >> 5)) >> (u & 31)) & 1u;
}

// Does row [s, e) hold a source in the frontier?  Lane-serial scan with early exit.
__device__ __forceinline__ bool scan_serial(const int32_t *__restrict__ colidx, int32_t s, int32_t e,
                                            const uint32_t *__restrict__ front) {
    for (int32_t i = s; i < e; ++i)
        if (in_front(front, __ldg(colidx + i))) return true;
    return false;
}

// Warp-cooperative scan of the rows flagged in `wm` (one at a time, early exit per chunk).
__device__ __forceinline__ bool scan_warp_rows(unsigned wm, int32_t s, int32_t e, const int32_t *__restrict__ colidx,
                                               const uint32_t *__restrict__ front, bool found) {
    const int lane = threadIdx.x & 31;
    while (wm) {
        const int l = __ffs(wm) - 1;
        wm &= wm - 1;
        const int32_t ws = __shfl_sync(0xffffffffu, s, l), we = __shfl_sync(0xffffffffu, e, l);
        bool hit = false;
        for (int32_t base = ws; base < we; base += 32) {
            const int32_t i = base + lane;
            const bool h = i < we && in_front(front, __ldg(colidx + i));
            if (__any_sync(0xffffffffu, h)) {
                hit = true;
                break;
            }
        }
        if (lane == l) found = hit;
    }
    return found;
}

__global__ void __launch_bounds__(BFS_THREADS) k_bfs_init(int32_t *level, uint32_t *visited, uint32_t *front,
                                                          int32_t V, int32_t nwords, int32_t source) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V; i += (int64_t)gridDim.x * blockDim.x)
        level[i] = (i == source) ? 0 : -1;
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bit = (w == (source >> 5)) ? (1u << (source & 31)) : 0u;
        visited[w] = bit;
        front[w] = bit;
    }
}

// Unblocked pull level.  next is written whole (one word per warp), visited updated,
// count accumulates the size of the new frontier.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_pull_level(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx, int32_t V,
                                                                int32_t nwords, const uint32_t *__restrict__ front,
                                                                uint32_t *__restrict__ next, uint32_t *visited,
                                                                int32_t *level, int32_t new_level,
                                                                unsigned long long *count,
                                                                const int32_t *__restrict__ out_rowptr) {
    __shared__ unsigned long long red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long found_total = 0, deg_total = 0;
    const int64_t nw = (int64_t)gridDim.x * BFS_WARPS;
    for (int64_t w = (int64_t)blockIdx.x * BFS_WARPS + warp; w < nwords; w += nw) {
        const uint32_t vis = visited[w];
        const int64_t v = w * 32 + lane;
        const bool cand = v < V && !((vis >> lane) & 1u);
        uint32_t nb = 0;
        if (__any_sync(0xffffffffu, cand)) {
            int32_t s = 0, e = 0;
            if (cand) {
                s = __ldg(rowptr + v);
                e = __ldg(rowptr + v + 1);
            }
            const int32_t deg = e - s;
            bool found = false;
            if (cand && deg < 32) found = scan_serial(colidx, s, e, front);
            found = scan_warp_rows(__ballot_sync(0xffffffffu, cand && deg >= 32), s, e, colidx, front, found);
            nb = __ballot_sync(0xffffffffu, found);
            if (found) {
                level[v] = new_level;
                deg_total += (unsigned long long)(__ldg(out_rowptr + v + 1) - __ldg(out_rowptr + v));
            }
            if (lane == 0 && nb) visited[w] = vis | nb;
        }
        if (lane == 0) {
            next[w] = nb;
            found_total += __popc(nb);
        }
    }
    const unsigned long long t = block_sum<unsigned long long>(found_total, red);
    const unsigned long long dt = block_sum<unsigned long long>(deg_total, red);
    if (threadIdx.x == 0 && t) atomicAdd(count, t);
    if (threadIdx.x == 0 && dt) atomicAdd(count + 1, dt);
}

// TOCAB level, phase 1 (Alg. 4 form for traversal): local row r of the row space belongs to
// destination id_map[r]; bit r of rowbits = "some in-edge of r inside its block comes from
// the frontier", computed only for unvisited destinations.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_block_level(const int32_t *__restrict__ rowptr,
                                                                 const int32_t *__restrict__ colidx,
                                                                 const int32_t *__restrict__ id_map, int64_t R,
                                                                 const uint32_t *__restrict__ front,
                                                                 const uint32_t *__restrict__ visited,
                                                                 uint32_t *__restrict__ rowbits) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ngroups = (R + 31) >> 5;
    const int64_t nw = (int64_t)gridDim.x * BFS_WARPS;
    for (int64_t grp = (int64_t)blockIdx.x * BFS_WARPS + warp; grp < ngroups; grp += nw) {
        const int64_t r = grp * 32 + lane;
        bool cand = false;
        int32_t s = 0, e = 0;
        if (r < R) {
            const int32_t v = __ldg(id_map + r);
            cand = !((visited[v >> 5] >> (v & 31)) & 1u);
            if (cand) {
                s = __ldg(rowptr + r);
                e = __ldg(rowptr + r + 1);
            }
        }
        const int32_t deg = e - s;
        bool found = false;
        if (cand && deg < 32) found = scan_serial(colidx, s, e, front);
        found = scan_warp_rows(__ballot_sync(0xffffffffu, cand && deg >= 32), s, e, colidx, front, found);
        const uint32_t nb = __ballot_sync(0xffffffffu, found);
        if (lane == 0) rowbits[grp] = nb;
    }
}

// TOCAB level, phase 2 (the reduction of the local next arrays, Sec. 3.3, in the merge
// kernel of Fig. 5): CTA j owns vertices [j*k, (j+1)*k); it ORs the local bits of every
// block's slice of that range, then writes next, visited and levels for the range.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_merge(const uint32_t *__restrict__ rowbits,
                                                           const int32_t *__restrict__ id_map,
                                                           const int32_t *__restrict__ merge_off, int32_t B,
                                                           int32_t nranges, int32_t k, int32_t V, int32_t nwords,
                                                           uint32_t *__restrict__ next, uint32_t *visited,
                                                           int32_t *level, int32_t new_level,
                                                           unsigned long long *count,
                                                           const int32_t *__restrict__ out_rowptr) {
    extern __shared__ uint32_t hit[];  // k/32 words
    __shared__ unsigned long long red[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j = blockIdx.x;
    const int32_t vbase = j * k;
    const int kw = k >> 5;
    for (int t = threadIdx.x; t < kw; t += BFS_THREADS) hit[t] = 0u;
    __syncthreads();
    for (int32_t b = warp; b < B; b += BFS_WARPS) {
        const int32_t *o = merge_off + (int64_t)b * (nranges + 1) + j;
        const int32_t r0 = __ldg(o), r1 = __ldg(o + 1);
        for (int32_t r = r0 + lane; r < r1; r += 32) {
            if ((__ldg(rowbits + (r >> 5)) >> (r & 31)) & 1u) {
                const int32_t t = __ldg(id_map + r) - vbase;
                atomicOr(&hit[t >> 5], 1u << (t & 31));
            }
        }
    }
    __syncthreads();
    unsigned long long found_total = 0, deg_total = 0;
    for (int t = threadIdx.x; t < kw; t += BFS_THREADS) {
        const int64_t w = (int64_t)(vbase >> 5) + t;
        if (w >= nwords) break;
        const uint32_t vis = visited[w];
        const uint32_t nb = hit[t] & ~vis;
        next[w] = nb;
        if (nb) {
            visited[w] = vis | nb;
            found_total += __popc(nb);
            uint32_t m = nb;
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int64_t v = w * 32 + bit;
                level[v] = new_level;
                deg_total += (unsigned long long)(__ldg(out_rowptr + v + 1) - __ldg(out_rowptr + v));
            }
        }
    }
    const unsigned long long tot = block_sum<unsigned long long>(found_total, red);
    const unsigned long long dt = block_sum<unsigned long long>(deg_total, red);
    if (threadIdx.x == 0 && tot) atomicAdd(count, tot);
    if (threadIdx.x == 0 && dt) atomicAdd(count + 1, dt);
}

// Push (top-down, data-driven) levels for small frontiers (Sec. 3.3: the push phases of the
// push-pull-push schedule, Alg. 3 without sigma): every frontier vertex in the queue scans its
// out-edges; an unvisited neighbour is claimed with an atomic OR on the visited bitmap, gets
// its level, joins the next bitmap and is appended to the next queue (warp-aggregated).
// Edge-balanced push level: the out-degrees of the queue are scanned (pre[q+1]); thread t takes
// edges t, t + stride, ... of the frontier's concatenated out-rows, finds its row by binary
// search in pre, and claims the neighbour as above.  Hubs spread over the whole grid.
__global__ void k_push_degrees(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ queue, int32_t qn,
                               int32_t *deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < qn; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = queue[i];
        deg[i] = __ldg(rowptr + u + 1) - __ldg(rowptr + u);
    }
}

__global__ void __launch_bounds__(BFS_THREADS) k_bfs_push_edges(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx,
                                                                const int32_t *__restrict__ queue, int32_t qn,
                                                                const int64_t *__restrict__ pre, int64_t total,
                                                                uint32_t *visited, uint32_t *next, int32_t *level,
                                                                int32_t new_level, int32_t *next_queue,
                                                                unsigned long long *count) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < total; base += stride) {
        const int64_t e = base + lane;
        bool claimed = false;
        int32_t v = 0;
        if (e < total) {
            int32_t lo = 0, hi = qn;  // last i with pre[i] <= e
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (__ldg(pre + mid) <= e) lo = mid; else hi = mid;
            }
            const int32_t u = __ldg(queue + lo);
            v = __ldg(colidx + __ldg(rowptr + u) + (e - __ldg(pre + lo)));
            const uint32_t bit = 1u << (v & 31);
            if (!(visited[v >> 5] & bit)) {
                const uint32_t old = atomicOr(visited + (v >> 5), bit);
                claimed = !(old & bit);
            }
        }
        const unsigned cm = __ballot_sync(0xffffffffu, claimed);
        if (cm) {
            int32_t pos0 = 0;
            if (lane == __ffs(cm) - 1) pos0 = (int32_t)atomicAdd(count, (unsigned long long)__popc(cm));
            pos0 = __shfl_sync(0xffffffffu, pos0, __ffs(cm) - 1);
            unsigned long long dg = 0;
            if (claimed) {
                level[v] = new_level;
                atomicOr(next + (v >> 5), 1u << (v & 31));
                next_queue[pos0 + __popc(cm & ((1u << lane) - 1u))] = v;
                dg = (unsigned long long)(__ldg(rowptr + v + 1) - __ldg(rowptr + v));
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) dg += __shfl_xor_sync(0xffffffffu, dg, d);
            if (lane == 0 && dg) atomicAdd(count + 1, dg);
        }
    }
}

// ---- cluster-resident push levels ------------------------------------------------------------
// Consecutive push levels with small frontiers run inside ONE launch of a thread-block cluster:
// the cluster's hardware barrier (release/acquire at cluster scope) ends each level, so a level
// costs a few dependent memory round trips instead of a host round trip and five launches.  The
// grid is exactly one cluster, so every CTA is co-scheduled by construction and no CTA waits on
// anything but that barrier.
// Level L: the frontier is the concatenation of the C CTAs' queue segments of level L-1 (the
// host's vertex queue for the first level); CTA c expands the c-th slice of it in batches of
// RES_THREADS vertices, and a CTA-wide scan of the out-degrees deals the batch's edges out one
// per thread.  A neighbour is claimed by an atomic OR on visited, gets its level, and is appended
// (warp-aggregated, position from a shared-memory counter) to CTA c's own segment with its
// out-edge range, which the next level reads instead of the row offsets.  After the barrier
// warp 0 of every CTA reads all C counters through distributed shared memory; every thread then
// holds the same counts and takes the same decision, the host's: stop when the frontier is
// empty, when direction optimisation switches to pull (m_f > m_u / 14), or when the next level
// has more than `cap` vertices or out-edges.  At the end the segments are copied, in CTA order,
// into the host's queue for the next level.  Everything written during the launch by other CTAs
// is read with L2 loads (ld.global.cg), never through L1.
constexpr int RES_THREADS = 1024;
constexpr int RES_WARPS = RES_THREADS / 32;
constexpr int RES_MAX_CTAS = 16;

struct ResOut {  // written by CTA 0, thread 0 when the launch ends
    unsigned long long front;  // frontier size of level `lvl`
    double m_f, m_u;           // its out-edges, and those of the unvisited vertices
    int32_t lvl;               // the next level to expand
    int32_t levels;            // levels expanded by the launch
};

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Exclusive prefix sum over the CTA (RES_THREADS threads); *total gets the sum.  All threads call it.
__device__ __forceinline__ int32_t res_block_scan(int32_t x, int32_t *wsum /* [RES_WARPS + 1] */, int32_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = wsum[lane];
        int32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        wsum[lane] = wi - w;  // exclusive over warps
        if (lane == 31) wsum[RES_WARPS] = wi;
    }
    __syncthreads();
    *total = wsum[RES_WARPS];
    return wsum[warp] + inc - x;
}

// seg_v / seg_r: [2 parities][C CTAs][cap] vertex IDs and out-edge ranges of the claimed vertices.
__global__ void __launch_bounds__(RES_THREADS, 1) k_bfs_push_resident(
    const int32_t *__restrict__ rowptr, const int32_t *__restrict__ colidx, uint32_t *visited, int32_t *level,
    int32_t *q0, int32_t *q1, int32_t *seg_v, int2 *seg_r, int64_t *trace, int32_t lvl0, int32_t n0, double mf0,
    double mu0, int32_t cap, int32_t max_levels, ResOut *out) {
    namespace cgs = cooperative_groups;
    __shared__ int32_t sh_start[RES_THREADS], sh_off[RES_THREADS];
    __shared__ int32_t wsum[RES_WARPS + 1];
    __shared__ unsigned long long s_cnt[2][2];  // this CTA's claims by level parity: vertices, out-edges
    __shared__ int32_t s_pre[RES_MAX_CTAS + 1];  // prefix of the segment counts (the current frontier)
    __shared__ unsigned long long s_edges;       // out-edges of the current frontier
    cgs::cluster_group cluster = cgs::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t C = (int32_t)gridDim.x, c = (int32_t)blockIdx.x;
    if (tid < 4) s_cnt[tid >> 1][tid & 1] = 0ull;  // ordered before any claim by the scan's barriers
    int32_t lvl = lvl0, levels = 0, n = n0;
    double mf = mf0, mu = mu0;
    bool first = true;  // the frontier is the host's queue (first level), else the segments
    for (;;) {
        const int par = lvl & 1;  // claims of this level: counters s_cnt[par], segments of parity par
        if (!first && tid == 0) {  // read remotely before the previous barrier, by every CTA
            s_cnt[par][0] = 0ull;
            s_cnt[par][1] = 0ull;
        }
        const int32_t *hq = (lvl & 1) ? q1 : q0;
        const int2 *in_r = seg_r + (size_t)(par ^ 1) * C * cap;
        int32_t *out_v = seg_v + ((size_t)par * C + c) * cap;
        int2 *out_r = seg_r + ((size_t)par * C + c) * cap;
        const int32_t lo = (int32_t)((int64_t)n * c / C), hi = (int32_t)((int64_t)n * (c + 1) / C);
        for (int32_t b0 = lo; b0 < hi; b0 += RES_THREADS) {
            const int32_t i = b0 + tid;
            int32_t s = 0, e = 0;
            if (i < hi) {
                if (first) {
                    const int32_t u = __ldcg(hq + i);
                    s = __ldg(rowptr + u);
                    e = __ldg(rowptr + u + 1);
                } else {  // entry i of the concatenated segments
                    int32_t a = 0;
                    while (a + 1 < C && s_pre[a + 1] <= i) ++a;
                    const int2 r = __ldcg(in_r + (size_t)a * cap + (i - s_pre[a]));
                    s = r.x;
                    e = r.y;
                }
            }
            int32_t total;
            const int32_t off = res_block_scan(e - s, wsum, &total);
            sh_start[tid] = s;
            sh_off[tid] = off;
            __syncthreads();
            const int32_t nb = min(RES_THREADS, hi - b0);
            for (int32_t base = warp * 32; base < total; base += RES_THREADS) {
                const int32_t k = base + lane;
                bool claimed = false;
                int32_t v = 0, vs = 0, ve = 0;
                if (k < total) {  // the last vertex of the batch whose edges start at or before k
                    int32_t a = 0, z = nb - 1;
                    while (a < z) {
                        const int32_t mid = (a + z + 1) >> 1;
                        if (sh_off[mid] <= k) a = mid; else z = mid - 1;
                    }
                    v = __ldg(colidx + sh_start[a] + (k - sh_off[a]));
                    const uint32_t bit = 1u << (v & 31);
                    claimed = !(atomicOr(visited + (v >> 5), bit) & bit);
                }
                if (claimed) {
                    level[v] = lvl + 1;
                    vs = __ldg(rowptr + v);
                    ve = __ldg(rowptr + v + 1);
                }
                const unsigned cm = __ballot_sync(0xffffffffu, claimed);
                if (cm) {
                    const int leader = __ffs(cm) - 1;
                    unsigned long long dg = (unsigned long long)(ve - vs);
#pragma unroll
                    for (int d = 16; d > 0; d >>= 1) dg += __shfl_xor_sync(0xffffffffu, dg, d);
                    unsigned long long pos0 = 0;
                    if (lane == leader) {
                        pos0 = atomicAdd(&s_cnt[par][0], (unsigned long long)__popc(cm));
                        atomicAdd(&s_cnt[par][1], dg);
                    }
                    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
                    if (claimed) {
                        const unsigned long long p = pos0 + (unsigned)__popc(cm & ((1u << lane) - 1u));
                        if (p < (unsigned long long)cap) {  // always: a CTA claims at most the level's edges
                            out_v[p] = v;
                            out_r[p] = make_int2(vs, ve);
                        }
                    }
                }
            }
            __syncthreads();  // the batch's offsets are read before the next batch overwrites them
        }
        ++levels;
        cluster_barrier();
        if (warp == 0) {  // every CTA's counters of this level, through distributed shared memory
            unsigned long long cn = 0, ce = 0;
            if (lane < C) {
                const unsigned long long *rc = cluster.map_shared_rank(&s_cnt[par][0], (unsigned)lane);
                cn = rc[0];
                ce = rc[1];
            }
            unsigned long long inc = cn;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += y;
            }
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) ce += __shfl_xor_sync(0xffffffffu, ce, d);
            if (lane < C) s_pre[lane + 1] = (int32_t)inc;
            if (lane == 0) {
                s_pre[0] = 0;
                s_edges = ce;
            }
        }
        __syncthreads();
        n = s_pre[C];
        mf = (double)s_edges;
        mu -= mf;
        ++lvl;
        first = false;
        if (c == 0 && tid == 0 && lvl < TC_BFS_TRACE) trace[lvl] = n;
        if (n == 0 || mf > mu / 14.0 || n > cap || mf > (double)cap || levels >= max_levels) break;
    }
    // the frontier of level lvl into the host's queue for it, segments in CTA order
    {
        const int par = (lvl - 1) & 1;
        const int32_t *src = seg_v + ((size_t)par * C + c) * cap;
        int32_t *dst = ((lvl & 1) ? q1 : q0) + s_pre[c];
        const int32_t cnt = s_pre[c + 1] - s_pre[c];
        for (int32_t i = tid; i < cnt; i += RES_THREADS) dst[i] = __ldcg(src + i);
    }
    if (c == 0 && tid == 0) {
        out->front = (unsigned long long)n;
        out->m_f = mf;
        out->m_u = mu;
        out->lvl = lvl;
        out->levels = levels;
    }
    cluster_barrier();  // no CTA leaves while another may still read its shared memory
}

// front = the bits of the queue's vertices (the frontier bitmap after resident push levels).
__global__ void k_queue_bits(const int32_t *__restrict__ queue, int64_t qn, uint32_t *front) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < qn; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = queue[i];
        atomicOr(front + (v >> 5), 1u << (v & 31));
    }
}

// Cluster size for the resident push levels: 16 CTAs when the device schedules such a cluster
// of RES_THREADS-thread CTAs, else 8, else 0 (resident levels off).
static int res_cluster_size(cudaStream_t s) {
    static int chosen = -1;
    if (chosen >= 0) return chosen;
    chosen = 0;
    for (int C : {16, 8}) {
        if (C > 8 && cudaFuncSetAttribute(k_bfs_push_resident, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                         cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C);
        cfg.blockDim = dim3(RES_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_bfs_push_resident, &cfg) == cudaSuccess && nclusters >= 1) {
            chosen = C;
            break;
        }
        cudaGetLastError();
    }
    return chosen;
}

// Queue of the vertices set in a bitmap (for a push level after a pull level): per word a
// popcount, an exclusive scan (positions), then the write.
__global__ void k_bitmap_count(const uint32_t *bits, int32_t nwords, int32_t *cnt) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x)
        cnt[w] = __popc(bits[w]);
}

__global__ void k_bitmap_queue(const uint32_t *bits, int32_t nwords, const int64_t *pos, int32_t *queue) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t m = bits[w];
        int64_t p = pos[w];
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            queue[p++] = (int32_t)(w * 32 + b);
        }
    }
}

// edges_reached = sum of out-degrees of vertices with level >= 0; reached = their count.
__global__ void __launch_bounds__(BFS_THREADS) k_bfs_stats(const int32_t *level, const int32_t *out_rowptr, int32_t V,
                                                           unsigned long long *out) {
    __shared__ unsigned long long red[32];
    unsigned long long n = 0, m = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        if (level[v] >= 0) {
            ++n;
            m += (unsigned long long)(out_rowptr[v + 1] - out_rowptr[v]);
        }
    }
    n = block_sum<unsigned long long>(n, red);
    m = block_sum<unsigned long long>(m, red);
    if (threadIdx.x == 0) {
        atomicAdd(out, n);
        atomicAdd(out + 1, m);
    }
}

__global__ void k_set_int(int32_t *p, int32_t v) { *p = v; }

static int bfs_impl(const tc_graph *cg, const tc_part *part, int32_t source, const tc_bfs_params *bp,
                    int32_t *levels_out, tc_bfs_stats *stats, cudaStream_t s) {
    tc_graph *g = const_cast<tc_graph *>(cg);
    const int32_t V = g->V;
    const int32_t nwords = (V + 31) / 32;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    TC_TRY(g->ws_bits.alloc((size_t)nwords * 4 * 3 + 64));
    uint32_t *visited = g->ws_bits.as<uint32_t>();
    uint32_t *bufs[2] = {visited + nwords, visited + 2 * nwords};
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(visited + 3 * nwords + (nwords & 1));
    int32_t *level = levels_out;
    if (bp->out_mem == TC_MEM_HOST) {
        TC_TRY(g->ws_misc.alloc((size_t)V * 4 + 256));
        level = g->ws_misc.as<int32_t>();
    }
    const int grid = caps.sms * 8;
    float ms_total = 0;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (bp->profile) {
        TC_CUDA(cudaEventCreate(&ev[0]));
        TC_CUDA(cudaEventCreate(&ev[1]));
        TC_CUDA(cudaEventRecord(ev[0], s));
    }
    k_bfs_init<<<grid, BFS_THREADS, 0, s>>>(level, visited, bufs[0], V, nwords, source);
    TC_LAUNCH_CHECK();
    const bool can_push = bp->push_threshold > 0.0f;
    // push-level buffers live with the graph (no allocation, and so no synchronisation, per call)
    DevBuf &queues = g->ws_queue, &qcnt = g->ws_qcnt, &qpos = g->ws_qpos;
    int32_t *q[2] = {nullptr, nullptr};
    const int64_t cap = (int64_t)(V > nwords ? V : nwords) + 16;
    if (can_push) {
        TC_TRY(queues.alloc((size_t)2 * V * 4 + 64));
        TC_TRY(qcnt.alloc((size_t)cap * 4));
        TC_TRY(qpos.alloc((size_t)cap * 8));
        TC_TRY(g->ws_scan.alloc((size_t)(scan_ws_elems(cap) + 16) * 8));
        q[0] = queues.as<int32_t>();
        q[1] = q[0] + V;
        k_set_int<<<1, 1, 0, s>>>(q[0], source);
        TC_LAUNCH_CHECK();
    }
    bool have_queue = can_push;  // the queue q[lvl & 1] holds the current frontier
    unsigned long long front_count = 1;
    if (!g->h_counts) TC_CUDA(cudaMallocHost(&g->h_counts, 64));
    unsigned long long *h_cnt = g->h_counts;
    // resident push levels: one cluster runs consecutive push levels whose frontier has at most
    // res_cap vertices and out-edges (queue segments of res_cap entries per CTA and parity)
    const int32_t res_cap = bp->resident_edges < 0 ? TC_BFS_RESIDENT_DEFAULT : bp->resident_edges;
    const int res_C = (can_push && res_cap > 0) ? res_cluster_size(s) : 0;
    int32_t *res_v = nullptr;  // [2][res_C][res_cap] queue segments
    int2 *res_r = nullptr;     // their out-edge ranges
    int64_t *res_trace = nullptr;
    ResOut *res_out = nullptr;
    if (res_C > 0) {
        const size_t nseg = (size_t)2 * res_C * res_cap;
        TC_TRY(g->ws_res.alloc(nseg * 12 + 64 + TC_BFS_TRACE * 8 + 64));
        res_r = g->ws_res.as<int2>();
        res_v = reinterpret_cast<int32_t *>(res_r + nseg);
        res_out = reinterpret_cast<ResOut *>(reinterpret_cast<unsigned char *>(res_v + nseg) + 64 -
                                             (reinterpret_cast<uintptr_t>(res_v + nseg) & 63));
        res_trace = reinterpret_cast<int64_t *>(reinterpret_cast<unsigned char *>(res_out) + 64);
    }
    bool bits_valid = true;  // bufs[lvl & 1] holds the frontier (not after resident push levels)
    int resident_levels = 0;
    // direction switching (Beamer et al.): edges out of the frontier (m_f) against edges out of
    // unvisited vertices (m_u); push -> pull when m_f > m_u / 14, pull -> push when the
    // frontier holds fewer than push_threshold * V vertices
    int32_t sdeg[2] = {0, 0};
    TC_CUDA(cudaMemcpyAsync(sdeg, g->out_rowptr.as<int32_t>() + source, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    double m_f = (double)(sdeg[1] - sdeg[0]);
    double m_u = (double)g->E - m_f;
    bool pushing = can_push;
    int lvl = 0, tocab_levels = 0, push_levels = 0;
    int st = TC_OK;
    cudaEvent_t lev[2] = {nullptr, nullptr};
    if (bp->profile && stats) {
        TC_CUDA(cudaEventCreate(&lev[0]));
        TC_CUDA(cudaEventCreate(&lev[1]));
    }
    const size_t merge_smem = part ? (size_t)(part->k / 32) * 4 : 0;
    while (front_count > 0) {
        uint32_t *front = bufs[lvl & 1], *next = bufs[(lvl + 1) & 1];
        if (cudaMemsetAsync(cnt, 0, 16, s) != cudaSuccess) { st = fail(TC_ERR_CUDA, "memset failed"); break; }
        if (can_push) {
            if (pushing && m_f > m_u / 14.0) pushing = false;
            else if (!pushing && (double)front_count < (double)bp->push_threshold * (double)V) pushing = true;
        }
        const bool use_push = can_push && pushing;
        const bool use_tocab = !use_push && part && bp->tocab_threshold >= 0.0f &&
                               (double)front_count > (double)bp->tocab_threshold * (double)V;
        if (stats && lvl < TC_BFS_TRACE) {
            stats->level_kind[lvl] = use_push ? 2 : (use_tocab ? 1 : 0);
            stats->level_frontier[lvl] = (int64_t)front_count;
        }
        if (lev[0]) cudaEventRecord(lev[0], s);
        if (use_push && res_C > 0 && have_queue && (int64_t)front_count <= res_cap && m_f <= (double)res_cap) {
            // consecutive push levels in one cluster launch; the host reads where they stopped
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(res_C);
            cfg.blockDim = dim3(RES_THREADS);
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = res_C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, k_bfs_push_resident, (const int32_t *)g->out_rowptr.as<int32_t>(),
                                               (const int32_t *)g->out_colidx.as<int32_t>(), visited, level, q[0],
                                               q[1], res_v, res_r, res_trace, (int32_t)lvl, (int32_t)front_count,
                                               m_f, m_u, res_cap, (int32_t)(V + 1), res_out);
            if (lev[1] && e == cudaSuccess) e = cudaEventRecord(lev[1], s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt + 2, res_out, sizeof(ResOut), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { st = fail(TC_ERR_CUDA, "bfs resident levels from %d: %s", lvl, cudaGetErrorString(e)); break; }
            ResOut ro;
            memcpy(&ro, h_cnt + 2, sizeof(ro));
            if (ro.levels < 1 || ro.lvl != lvl + ro.levels) { st = fail(TC_ERR_CUDA, "bfs resident levels: bad exit state"); break; }
            if (stats) {
                float seg_ms = 0.0f;
                if (lev[1]) cudaEventElapsedTime(&seg_ms, lev[0], lev[1]);
                const int hi = ro.lvl < TC_BFS_TRACE ? ro.lvl : TC_BFS_TRACE;
                if (lvl + 1 < hi) {
                    e = cudaMemcpy(stats->level_frontier + lvl + 1, res_trace + lvl + 1, (size_t)(hi - lvl - 1) * 8,
                                   cudaMemcpyDeviceToHost);
                    if (e != cudaSuccess) { st = fail(TC_ERR_CUDA, "bfs trace copy: %s", cudaGetErrorString(e)); break; }
                }
                for (int l = lvl; l < hi; ++l) {
                    stats->level_kind[l] = 3;
                    stats->level_ms[l] = seg_ms / (float)ro.levels;
                }
            }
            push_levels += ro.levels;
            resident_levels += ro.levels;
            front_count = ro.front;
            m_f = ro.m_f;
            m_u = ro.m_u;
            lvl = ro.lvl;
            have_queue = true;
            bits_valid = false;
            continue;
        }
        if (!use_push && !bits_valid) {  // pull levels read the frontier bitmap: rebuild it from the queue
            if (cudaMemsetAsync(front, 0, (size_t)nwords * 4, s) != cudaSuccess) { st = fail(TC_ERR_CUDA, "memset failed"); break; }
            k_queue_bits<<<grid, BFS_THREADS, 0, s>>>(q[lvl & 1], (int64_t)front_count, front);
            if (cudaGetLastError() != cudaSuccess) { st = fail(TC_ERR_CUDA, "launch failed"); break; }
        }
        bits_valid = true;
        push_levels += use_push ? 1 : 0;
        if (use_push) {
            if (!have_queue) {  // frontier came from a pull level: bitmap -> queue
                k_bitmap_count<<<grid, BFS_THREADS, 0, s>>>(front, nwords, qcnt.as<int32_t>());
                if (cudaGetLastError() != cudaSuccess) { st = fail(TC_ERR_CUDA, "launch failed"); break; }
                st = scan_i32_to_i64_ws(qcnt.as<int32_t>(), nwords, qpos.as<int64_t>(), g->ws_scan.as<int64_t>(), s);
                if (st != TC_OK) break;
                k_bitmap_queue<<<grid, BFS_THREADS, 0, s>>>(front, nwords, qpos.as<int64_t>(), q[lvl & 1]);
            }
            if (cudaMemsetAsync(next, 0, (size_t)nwords * 4, s) != cudaSuccess) { st = fail(TC_ERR_CUDA, "memset failed"); break; }
            // out-degree prefix of the queue: frontier edges m_f are already known on the host
            const int32_t qn = (int32_t)front_count;
            k_push_degrees<<<grid, BFS_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), q[lvl & 1], qn,
                                                        qcnt.as<int32_t>());
            if (cudaGetLastError() != cudaSuccess) { st = fail(TC_ERR_CUDA, "launch failed"); break; }
            st = scan_i32_to_i64_ws(qcnt.as<int32_t>(), qn, qpos.as<int64_t>(), g->ws_scan.as<int64_t>(), s);
            if (st != TC_OK) break;
            const int64_t total = (int64_t)(m_f + 0.5);
            if (total > 0)
                k_bfs_push_edges<<<grid, BFS_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(),
                                                              q[lvl & 1], qn, qpos.as<int64_t>(), total, visited, next,
                                                              level, lvl + 1, q[(lvl + 1) & 1], cnt);
            have_queue = true;
        } else if (use_tocab) {
            k_bfs_block_level<<<grid, BFS_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                           part->id_map.as<int32_t>(), part->R, front, visited,
                                                           part->rowbits.as<uint32_t>());
            k_bfs_merge<<<part->nranges, BFS_THREADS, merge_smem, s>>>(part->rowbits.as<uint32_t>(),
                                                                       part->id_map.as<int32_t>(),
                                                                       part->merge_off.as<int32_t>(), part->B,
                                                                       part->nranges, part->k, V, nwords, next,
                                                                       visited, level, lvl + 1, cnt,
                                                                       g->out_rowptr.as<int32_t>());
            ++tocab_levels;
            have_queue = false;
        } else {
            k_bfs_pull_level<<<grid, BFS_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), V,
                                                          nwords, front, next, visited, level, lvl + 1, cnt,
                                                          g->out_rowptr.as<int32_t>());
            have_queue = false;
        }
        if (lev[1]) cudaEventRecord(lev[1], s);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt, cnt, 16, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { st = fail(TC_ERR_CUDA, "bfs level %d: %s", lvl, cudaGetErrorString(e)); break; }
        front_count = h_cnt[0];
        m_f = (double)h_cnt[1];
        m_u -= m_f;
        if (lev[1] && lvl < TC_BFS_TRACE) cudaEventElapsedTime(&stats->level_ms[lvl], lev[0], lev[1]);
        ++lvl;
    }
    if (lev[0]) {
        cudaEventDestroy(lev[0]);
        cudaEventDestroy(lev[1]);
    }
    TC_TRY(st);
    if (bp->profile) {
        TC_CUDA(cudaEventRecord(ev[1], s));
        TC_CUDA(cudaEventSynchronize(ev[1]));
        TC_CUDA(cudaEventElapsedTime(&ms_total, ev[0], ev[1]));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (stats) {
        TC_CUDA(cudaMemsetAsync(cnt, 0, 16, s));
        k_bfs_stats<<<grid, BFS_THREADS, 0, s>>>(level, g->out_rowptr.as<int32_t>(), V, cnt);
        TC_LAUNCH_CHECK();
        unsigned long long hs[2];
        TC_CUDA(cudaMemcpyAsync(hs, cnt, 16, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        stats->levels = lvl;
        stats->tocab_levels = tocab_levels;
        stats->push_levels = push_levels;
        stats->resident_levels = resident_levels;
        stats->reached = (int64_t)hs[0];
        stats->edges_reached = (int64_t)hs[1];
        stats->ms_total = ms_total;
    }
    if (bp->out_mem == TC_MEM_HOST) {
        TC_CUDA(cudaMemcpyAsync(levels_out, level, (size_t)V * 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
    }
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_bfs_pull(const tc_graph *g, const tc_part *part, int32_t source, const tc_bfs_params *params,
                           int32_t *levels_out, tc_bfs_stats *stats, void *stream) {
    using namespace tc;
    if (!g || !params || !levels_out) return fail(TC_ERR_INVALID_ARG, "tc_bfs_pull: null graph, params or output");
    if (source < 0 || source >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_bfs_pull: source outside [0, V)");
    if (params->out_mem != TC_MEM_HOST && params->out_mem != TC_MEM_DEVICE)
        return fail(TC_ERR_INVALID_ARG, "tc_bfs_pull: bad out_mem");
    if (part && (part->g != g || part->dir != TC_PULL))
        return fail(TC_ERR_INVALID_ARG, "tc_bfs_pull: partition must be a TC_PULL partition of this graph");
    if (params->resident_edges > TC_BFS_RESIDENT_MAX)
        return fail(TC_ERR_INVALID_ARG, "tc_bfs_pull: resident_edges above %d", TC_BFS_RESIDENT_MAX);
    if (part && part->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_bfs_pull: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if (stats) memset(stats, 0, sizeof(*stats));
    return bfs_impl(g, part, source, params, levels_out, stats, (cudaStream_t)stream);
}
