// Topology-driven pull BFS with bitmap status arrays (Sec. 3.3, Fig. 1e/f).
//   unblocked level : warp per 32 vertices (one bitmap word); every unvisited vertex scans
//                     its in-edges with early exit until it finds a frontier source.
//   TOCAB level     : per block, a local "next" bit per local row (rows are scanned only
//                     over the block's sources), then a merge kernel ORs the local bits of
//                     all blocks per vertex range and writes levels, next and visited.
// Levels run TOCAB only when the frontier exceeds a fraction of V (Sec. 3.3).
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
    if (!g->h_counts) TC_CUDA(cudaMallocHost(&g->h_counts, 16));
    unsigned long long *h_cnt = g->h_counts;
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
    if (part && part->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_bfs_pull: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if (stats) memset(stats, 0, sizeof(*stats));
    return bfs_impl(g, part, source, params, levels_out, stats, (cudaStream_t)stream);
}
