// Many independent graphs in one batch: pull PageRank (Alg. 1) on the disjoint union of the
// graphs, every graph with its own teleport term (1-d)/V_g and its own dangling mass D_g.
// All iterations run in ONE persistent cooperative kernel (grid barrier between iterations,
// with a bounded spin) that is captured once into a CUDA graph and replayed.  The mapping of
// lanes to vertices (1, 4, 8 or 32 lanes per vertex, or the thread/warp hybrid) is a template
// parameter; tc_multi_autotune times every variant on the batch and keeps the fastest.
// A further variant (TC_MULTI_RESIDENT) keeps each graph inside one CTA for all iterations:
// the graph's contributions live in shared memory (compacted to its non-dangling vertices,
// 16-bit source indices), so no grid barrier and no L2 gather is needed; CTAs take graphs
// from a queue, largest first.  Inside the CTA the graph's in-edges are split evenly over the
// warps (head bits mark row starts), so skewed degrees leave no lane idle.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "tc_common_dev.cuh"

namespace tc {

constexpr int MU_THREADS = 256;
constexpr int MU_WARPS = MU_THREADS / 32;
constexpr int MU_CHUNK = 512;                  // vertices per warp work item
constexpr double MU_FX = 2305843009213693952.0;  // 2^61 fixed point: a graph's mass is <= 1
constexpr int MU_NVARIANTS = 6;
static const int kLanes[MU_NVARIANTS] = {-1, 1, 4, 8, 32, TC_MULTI_RESIDENT};  // -1: thread/warp hybrid
constexpr int MR_THREADS = 1024;                 // resident variant: one CTA per graph at a time

}  // namespace tc

struct tc_multigraph {
    tc_graph *g = nullptr;                 // the disjoint union
    int32_t n = 0;                         // graphs
    tc::DevBuf vtx_off, gid, invVg;        // int32[n+1], int32[V], float[n]
    tc::DevBuf rank, contrib, dacc, sync;  // float[V], float[2V], u64[3n], barrier words
    int32_t tuned_lanes = 0;               // 0: not tuned yet
    // resident variant (built on first use): compact index of every non-dangling vertex inside
    // its graph, in-edges as 16-bit compact sources, graph queue (largest first)
    bool res_built = false, res_ok = false;
    int32_t res_max = 0;                   // largest non-dangling count of a graph
    // the in-edge stream: every row's compact sources (uint16), one placeholder edge for an
    // empty row, padded to whole chunks; a head bit at every row's first edge; heads before every
    // 512-edge chunk; every graph's first stream edge; the row sums of one iteration (by vertex)
    tc::DevBuf cpos, src16, heads, hpre, eoff, order, scratch;
    // captured CUDA graph of the persistent launch, for one parameter set
    cudaGraphExec_t exec = nullptr;
    float cached_damping = -1.0f;
    int32_t cached_iters = -1, cached_drop = -1, cached_lanes = 0, cached_ctas = 0;
    ~tc_multigraph() {
        if (exec) cudaGraphExecDestroy(exec);
        delete g;
    }
};

namespace tc {

struct MultiArgs {
    const int32_t *rowptr, *colidx, *gid;
    const float *inv_outdeg, *invVg;
    int32_t V, n, iters, drop;
    float damping;
    float *contrib;             // [2][Vp]
    int64_t Vp;
    float *rank;                // [V]
    unsigned long long *dacc;   // [3][n]
    unsigned *bar;              // [0] count, [1] generation
    int *err;
};

// Grid-wide barrier with a bounded spin (about a second); on a timeout it records code 4.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == gridDim.x - 1) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > (1LL << 31)) {
                    atomicCAS(err, 0, 4);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = (*(volatile int *)err == 0);
    }
    __syncthreads();
    return ok != 0;
}

// Sum of the in-edges of vertex v over `lanes` cooperating lanes (sub = lane index in group).
template <int LANES>
__device__ __forceinline__ float gather_sum(const MultiArgs &a, const float *__restrict__ c, int64_t v, int sub,
                                            bool valid) {
    float acc = 0.0f;
    if (valid) {
        const int32_t s = __ldg(a.rowptr + v), e = __ldg(a.rowptr + v + 1);
        for (int32_t i = s + sub; i < e; i += LANES) acc += __ldg(c + __ldg(a.colidx + i));
    }
#pragma unroll
    for (int d = LANES / 2; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    return acc;
}

// Hybrid: a lane per vertex, rows of 32+ edges by the whole warp.
__device__ __forceinline__ float gather_hybrid(const MultiArgs &a, const float *__restrict__ c, int64_t v, bool valid) {
    const int lane = threadIdx.x & 31;
    int32_t s = 0, e = 0;
    if (valid) {
        s = __ldg(a.rowptr + v);
        e = __ldg(a.rowptr + v + 1);
    }
    float sum = 0.0f;
    if (e - s < 32)
        for (int32_t i = s; i < e; ++i) sum += __ldg(c + __ldg(a.colidx + i));
    unsigned wm = __ballot_sync(0xffffffffu, valid && e - s >= 32);
    while (wm) {
        const int l = __ffs(wm) - 1;
        wm &= wm - 1;
        const int32_t ws = __shfl_sync(0xffffffffu, s, l), we = __shfl_sync(0xffffffffu, e, l);
        float acc = 0.0f;
        for (int32_t i = ws + lane; i < we; i += 32) acc += __ldg(c + __ldg(a.colidx + i));
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == l) sum = acc;
    }
    return sum;
}

// Flush a lane's dangling sum for graph g (fixed point); lanes of a warp that share g are
// added first so that a warp issues one atomic per graph.
__device__ __forceinline__ void flush_dangling(unsigned long long *dn, int32_t g, float val, bool has) {
    const unsigned active = __ballot_sync(0xffffffffu, has);
    if (!active) return;
    const unsigned peers = __match_any_sync(0xffffffffu, has ? g : -1);
    unsigned long long fx = has ? (unsigned long long)__double2ll_rn((double)val * MU_FX) : 0ull;
    // sum over peers: every lane adds the values of its peers (at most 32 shuffles)
    unsigned long long tot = 0ull;
    unsigned m = peers;
    while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        tot += __shfl_sync(peers, fx, l);
    }
    const int lane = threadIdx.x & 31;
    if (has && (__ffs(peers) - 1) == lane && tot) atomicAdd(dn + g, tot);
}

// LANES: lanes per vertex (1, 4, 8, 32), or 0 for the hybrid.
template <int LANES>
__global__ void __launch_bounds__(MU_THREADS) k_multi_pagerank(MultiArgs a) {
    const int lane = threadIdx.x & 31;
    constexpr int L = LANES == 0 ? 1 : LANES;     // lanes per vertex in this warp step
    constexpr int VPW = 32 / L;                   // vertices per warp step
    const int sub = lane % L, slot = lane / L;
    const int64_t nitems = ((int64_t)a.V + MU_CHUNK - 1) / MU_CHUNK;
    const int64_t gw = (int64_t)blockIdx.x * MU_WARPS + (threadIdx.x >> 5);
    const int64_t nw = (int64_t)gridDim.x * MU_WARPS;
    unsigned long long *D[3] = {a.dacc, a.dacc + a.n, a.dacc + 2 * a.n};

    // ---- init: r0 = 1/V_g, contributions, D_0 per graph; D[1] cleared ----
    if (blockIdx.x == 0)
        for (int32_t g = threadIdx.x; g < a.n; g += MU_THREADS) D[1][g] = 0ull;
    for (int64_t it = gw; it < nitems; it += nw) {
        const int64_t v0 = it * MU_CHUNK;
        int32_t gcur = -1;
        float dl = 0.0f;
        for (int64_t v = v0 + lane; v < v0 + MU_CHUNK; v += 32) {
            const bool valid = v < a.V;
            const int32_t g = valid ? __ldg(a.gid + v) : -1;
            float r = 0.0f, inv = 1.0f;
            if (valid) {
                r = __ldg(a.invVg + g);
                inv = __ldg(a.inv_outdeg + v);
                a.contrib[v] = r * inv;
                if (a.iters == 0) a.rank[v] = r;
            }
            const bool change = __any_sync(0xffffffffu, g != gcur && gcur >= 0);
            if (change) {
                flush_dangling(D[0], gcur, dl, gcur >= 0 && dl != 0.0f);
                dl = 0.0f;
            }
            gcur = valid ? g : gcur;
            if (valid && inv == 0.0f) dl += r;
        }
        flush_dangling(D[0], gcur, dl, gcur >= 0 && dl != 0.0f);
    }
    if (!grid_barrier(a.bar, a.err)) return;

    for (int32_t iter = 0; iter < a.iters; ++iter) {
        const float *cur = a.contrib + (iter & 1) * a.Vp;
        float *nxt = a.contrib + ((iter + 1) & 1) * a.Vp;
        const unsigned long long *Dc = D[iter % 3];
        unsigned long long *Dn = D[(iter + 1) % 3];
        if (blockIdx.x == 0)
            for (int32_t g = threadIdx.x; g < a.n; g += MU_THREADS) D[(iter + 2) % 3][g] = 0ull;
        const bool last = iter == a.iters - 1;
        for (int64_t it = gw; it < nitems; it += nw) {
            const int64_t v0 = it * MU_CHUNK;
            const int64_t v1 = (v0 + MU_CHUNK < a.V) ? v0 + MU_CHUNK : a.V;
            int32_t gcur = -1;
            float dl = 0.0f;
            for (int64_t vb = v0; vb < v1; vb += VPW) {
                const int64_t v = vb + slot;
                const bool valid = v < v1;
                float sum;
                if (LANES == 0) sum = gather_hybrid(a, cur, v, valid);
                else sum = gather_sum<L>(a, cur, v, sub, valid);
                int32_t g = -1;
                float r = 0.0f, inv = 1.0f;
                if (valid && sub == 0) {
                    g = __ldg(a.gid + v);
                    const float ivg = __ldg(a.invVg + g);
                    const float spread = a.drop ? 0.0f : (float)((double)Dc[g] / MU_FX) * ivg;
                    r = (1.0f - a.damping) * ivg + a.damping * (sum + spread);
                    inv = __ldg(a.inv_outdeg + v);
                    nxt[v] = r * inv;
                    if (last) a.rank[v] = r;
                }
                const bool lead = valid && sub == 0;
                const bool change = __any_sync(0xffffffffu, lead && g != gcur && gcur >= 0);
                if (change) {
                    flush_dangling(Dn, gcur, dl, gcur >= 0 && dl != 0.0f);
                    dl = 0.0f;
                    gcur = -1;
                }
                if (lead) {
                    gcur = g;
                    if (inv == 0.0f) dl += r;
                }
            }
            flush_dangling(Dn, gcur, dl, gcur >= 0 && dl != 0.0f);
        }
        if (!grid_barrier(a.bar, a.err)) return;
    }
}

// ---- resident variant -----------------------------------------------------------------------
constexpr int MR_WARPS = MR_THREADS / 32;
constexpr int MR_CHUNK = 512;  // edges per warp chunk: 16 consecutive stream edges per lane
constexpr int MR_VB = 4;       // vertex groups per warp and step of the update

struct ResArgs {
    const uint16_t *src16;      // the in-edge stream: compact sources inside the graph; an empty
                                // row has one edge from the graph's zero slot (its non-dangling count)
    const uint16_t *heads;      // bit i of heads[q]: stream edge 16q + i is the first of its row
    const int32_t *hpre;        // [chunks] heads before stream edge 512c = rows started before it
    const int32_t *eoff;        // [n+1] first stream edge of every graph
    const int32_t *cpos;        // [V+1] exclusive count of non-dangling vertices before v
    const int32_t *vtx_off, *order;
    const float *inv_outdeg;
    int32_t n, iters, drop;
    float damping;
    float *sums;                // [V] in-edge sums of one iteration
    float *rank;                // [V]
    unsigned *next;             // queue counter
};

// One warp sums the rows of the stream edges [es, ee) over the contributions in shared memory
// (the in-edge sum of Alg. 1, edge-balanced): 16 consecutive edges per lane and chunk, a row
// break at every head bit.  Every vertex owns one row, so the k-th head is vertex k: rows that
// start in the range are written to a.sums[vertex] (rs = heads before es); the piece of the row
// already open at es is returned to the caller, which adds it once every warp has finished
// (rows may cross warp ranges).
__device__ __forceinline__ float res_walk(const ResArgs &a, const float *cs, int32_t es, int32_t ee, int32_t rs) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    int32_t rowbase = rs;  // rank of the row started by the next head
    float carry = 0.0f;    // value of the open row rowbase - 1 so far
    bool open = false;     // whether row rowbase - 1 started inside [es, ee)
    float lead = 0.0f;     // the open row's piece before the range's first head
    if (es >= ee) return 0.0f;
    const int32_t qb = es & ~(MR_CHUNK - 1);
    // software pipeline: the next chunk's sources and heads are loaded before this one is summed
    uint4 nc0, nc1;
    uint32_t nh;
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(a.src16 + qb + 16 * lane);
        nc0 = __ldg(p);
        nc1 = __ldg(p + 1);
        nh = __ldg(a.heads + (qb >> 4) + lane);
    }
    for (int32_t q0 = qb; q0 < ee; q0 += MR_CHUNK) {
        const uint4 c0 = nc0, c1 = nc1;
        uint32_t hd = nh;
        if (q0 + MR_CHUNK < ee) {
            const uint4 *p = reinterpret_cast<const uint4 *>(a.src16 + q0 + MR_CHUNK + 16 * lane);
            nc0 = __ldg(p);
            nc1 = __ldg(p + 1);
            nh = __ldg(a.heads + ((q0 + MR_CHUNK) >> 4) + lane);
        }
        const uint32_t words[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        float val[16];
        if (q0 >= es && q0 + MR_CHUNK <= ee) {  // whole chunk inside the range (warp-uniform)
#pragma unroll
            for (int i = 0; i < 16; ++i) val[i] = cs[(words[i >> 1] >> (16 * (i & 1))) & 0xFFFFu];
        } else {
            const int32_t e0 = q0 + 16 * lane;  // valid edges of this lane: [max(es, e0), min(ee, e0 + 16))
            const int32_t lo_i = es - e0, hi_i = ee - e0;
            uint32_t valid = 0xFFFFu;
            if (lo_i > 0) valid = lo_i >= 16 ? 0u : (valid & (0xFFFFu << lo_i));
            if (hi_i < 16) valid = hi_i <= 0 ? 0u : (valid & ((1u << hi_i) - 1u));
            hd &= valid;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t col = (words[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                val[i] = ((valid >> i) & 1u) ? cs[col] : 0.0f;
            }
        }
        // heads in earlier lanes and in the whole chunk, from bit-sliced ballots of the counts
        const int nh_l = __popc(hd);
        int before = 0, total = 0;
#pragma unroll
        for (int bit = 0; bit < 5; ++bit) {
            const uint32_t m = __ballot_sync(0xffffffffu, (nh_l >> bit) & 1);
            before += __popc(m & lt_mask) << bit;
            total += __popc(m) << bit;
        }
        // the lane's 16 edges: every head after the lane's first closes a whole row (rank
        // rowbase + before + j), the piece before its first head goes to the carry scan
        float seg = 0.0f, first = 0.0f;
        int32_t orow = rowbase + before;
        const uint32_t close_m = hd & (hd - 1u);
        const uint32_t first_m = hd & (0u - hd);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if ((close_m >> i) & 1u) a.sums[orow++] = seg;
            if ((first_m >> i) & 1u) first = seg;
            seg = ((hd >> i) & 1u) ? val[i] : seg + val[i];
        }
        const bool seen = hd != 0u;
        if (!seen) first = seg;
        // the open row's value across lanes: segmented inclusive scan, flags from one ballot
        const uint32_t F = __ballot_sync(0xffffffffu, seen);
        float v = seg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float vp = __shfl_up_sync(0xffffffffu, v, d);
            const int lo = lane - d + 1;
            const uint32_t win = lo > 0 ? (F >> lo) & ((1u << d) - 1u) : F & ((2u << lane) - 1u);
            if (lane >= d && win == 0u) v += vp;
        }
        const bool f = (F & ((2u << lane) - 1u)) != 0u;
        const float vprev = __shfl_up_sync(0xffffffffu, v, 1);
        const bool fprev = (F & lt_mask) != 0u;
        const float xprev = (lane == 0) ? carry : (fprev ? vprev : carry + vprev);
        const float closed = xprev + first;  // the row closed at the lane's first head
        if (seen && (before > 0 || open)) a.sums[rowbase + before - 1] = closed;
        if (!open && total > 0) lead = __shfl_sync(0xffffffffu, closed, __ffs(F) - 1);
        carry = __shfl_sync(0xffffffffu, f ? v : carry + v, 31);
        if (total > 0) open = true;
        rowbase += total;
    }
    if (!open) return carry;  // no head in the range: all of it belongs to the row open at es
    if (lane == 0) a.sums[rowbase - 1] = carry;
    return lead;
}

// CTA-wide sum of one float per thread, returned to every thread (fixed order: deterministic).
__device__ __forceinline__ float res_block_sum(float x, float *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    __syncthreads();  // red may still be read from the previous call
    if (lane == 0) red[warp] = x;
    __syncthreads();
    float t = lane < MR_WARPS ? red[lane] : 0.0f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
    return t;
}

// One CTA runs all iterations of a graph (Alg. 1 with the graph's own teleport and dangling
// mass), then takes the next graph of the queue.  The contributions of the graph's
// non-dangling vertices stay in shared memory.  An iteration: every warp sums an equal share
// of the graph's in-edges into a.sums; one warp adds the pieces of rows that cross warp
// ranges, in warp order; then a lane per vertex applies the update of Alg. 1 and overwrites its
// contribution in place (all sums are complete by then, so this is still a Jacobi step).
__global__ void __launch_bounds__(MR_THREADS, 1) k_multi_resident(ResArgs a) {
    extern __shared__ __align__(16) float cs[];
    __shared__ float red[32];
    __shared__ float lead[MR_WARPS];
    __shared__ int32_t lrow[MR_WARPS];
    __shared__ int32_t gnext;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (;;) {
        if (tid == 0) gnext = (int32_t)atomicAdd(a.next, 1u);
        __syncthreads();
        const int32_t gi = gnext;
        __syncthreads();
        if (gi >= a.n) break;
        const int32_t g = a.order[gi];
        const int32_t v0 = a.vtx_off[g], v1 = a.vtx_off[g + 1];
        const int32_t nv = v1 - v0;
        if (nv <= 0) continue;
        const int32_t c0 = a.cpos[v0];
        const float ivg = 1.0f / (float)nv;
        // this warp's share of the graph's stream edges, and rs = heads before its first edge
        const int32_t E0 = __ldg(a.eoff + g), ne = __ldg(a.eoff + g + 1) - E0;
        const int32_t per = ((ne + MR_WARPS - 1) / MR_WARPS + 15) & ~15;
        const int32_t es = E0 + min(warp * per, ne), ee = E0 + min((warp + 1) * per, ne);
        int32_t rs;
        {
            const int32_t qb = es & ~(MR_CHUNK - 1);
            const uint32_t h = __ldg(a.heads + (qb >> 4) + lane);
            const int32_t below = es - (qb + 16 * lane);  // edges of this lane before es
            const uint32_t m = below >= 16 ? 0xFFFFu : (below <= 0 ? 0u : (1u << below) - 1u);
            rs = __ldg(a.hpre + (qb >> 9)) + __reduce_add_sync(0xffffffffu, __popc(h & m));
            const uint32_t hes = __shfl_sync(0xffffffffu, h, (es - qb) >> 4);
            if (lane == 0) lrow[warp] = (es < ee && !((hes >> ((es - qb) & 15)) & 1u)) ? rs - 1 : -1;
        }
        // r0 = 1/V_g: contributions and the dangling mass; the zero slot after them
        if (tid == 0) cs[a.cpos[v1] - c0] = 0.0f;
        float dl = 0.0f;
        for (int32_t v = v0 + tid; v < v1; v += MR_THREADS) {
            const float inv = __ldg(a.inv_outdeg + v);
            if (inv == 0.0f) dl += ivg;
            else cs[__ldg(a.cpos + v) - c0] = ivg * inv;
            if (a.iters == 0) a.rank[v] = ivg;
        }
        float D = res_block_sum(dl, red);
        __syncthreads();
        for (int32_t it = 0; it < a.iters; ++it) {
            const bool last = it == a.iters - 1;
            const float spread = a.drop ? 0.0f : D * ivg;
            const float tele = (1.0f - a.damping) * ivg;
            const float lv = res_walk(a, cs, es, ee, rs);
            if (lane == 0) lead[warp] = lv;
            __syncthreads();
            if (warp == 0) {  // rows crossing warp ranges: the later pieces, in warp order
                const int32_t lr = lrow[lane];
                if (lr >= 0 && (lane == 0 || lrow[lane - 1] != lr)) {
                    float acc = 0.0f;
                    for (int w = lane; w < MR_WARPS && lrow[w] == lr; ++w) acc += lead[w];
                    a.sums[lr] += acc;
                }
            }
            __syncthreads();
            dl = 0.0f;
            // MR_VB groups of 32 vertices per warp and step: their loads are issued together
            for (int32_t vb = v0 + warp * 32; vb < v1; vb += MR_VB * MR_THREADS) {
                float inv[MR_VB], sum[MR_VB];
                int32_t cb[MR_VB];
#pragma unroll
                for (int k = 0; k < MR_VB; ++k) {
                    const int32_t gb = vb + k * MR_THREADS, v = gb + lane;
                    inv[k] = 0.0f;
                    sum[k] = 0.0f;
                    cb[k] = 0;
                    if (v < v1) {
                        inv[k] = __ldg(a.inv_outdeg + v);
                        sum[k] = a.sums[v];
                    }
                    if (gb < v1) cb[k] = __ldg(a.cpos + gb) - c0;
                }
#pragma unroll
                for (int k = 0; k < MR_VB; ++k) {
                    const int32_t v = vb + k * MR_THREADS + lane;
                    const bool valid = v < v1;
                    const float r = tele + a.damping * (sum[k] + spread);
                    const uint32_t nd = __ballot_sync(0xffffffffu, valid && inv[k] != 0.0f);
                    if (valid) {
                        if (inv[k] == 0.0f) dl += r;
                        else cs[cb[k] + __popc(nd & lt_mask)] = r * inv[k];
                        if (last) a.rank[v] = r;
                    }
                }
            }
            D = res_block_sum(dl, red);  // its barriers order the new contributions and sums
        }
    }
}

__global__ void k_multi_nondangling(const float *inv_outdeg, int32_t V, int32_t *flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = inv_outdeg[v] != 0.0f ? 1 : 0;
}

__global__ void k_multi_gid(const int32_t *vtx_off, int32_t n, int32_t V, int32_t *gid, float *invVg) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t lo = 0, hi = n;  // last g with vtx_off[g] <= v
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (vtx_off[mid] <= v) lo = mid; else hi = mid;
        }
        gid[v] = lo;
    }
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t nv = vtx_off[g + 1] - vtx_off[g];
        invVg[g] = nv > 0 ? 1.0f / (float)nv : 0.0f;
    }
}

// every in-edge u -> v must join two vertices of the same graph
__global__ void k_multi_check(const int32_t *rowptr, const int32_t *colidx, const int32_t *gid, int32_t V, int *bad) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = gid[v];
        for (int32_t i = rowptr[v]; i < rowptr[v + 1]; ++i)
            if (gid[colidx[i]] != g) {
                atomicOr(bad, 1);
                break;
            }
    }
}

__global__ void k_multi_graph_sizes(const int32_t *vtx_off, int32_t n, const int32_t *cpos, const int32_t *in_rowptr,
                                    int32_t *ndang_free, int32_t *edges) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
        ndang_free[g] = cpos[vtx_off[g + 1]] - cpos[vtx_off[g]];
        edges[g] = in_rowptr[vtx_off[g + 1]] - in_rowptr[vtx_off[g]];
    }
}

__global__ void k_multi_cpos_end(int32_t *cpos, const int32_t *flag, int32_t V) {
    cpos[V] = V > 0 ? cpos[V - 1] + flag[V - 1] : 0;
}

__global__ void k_res_empty(const int32_t *rowptr, int32_t V, int32_t *flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        flag[v] = rowptr[v + 1] == rowptr[v] ? 1 : 0;
}

// first stream edge of every graph (g = n: the stream's length)
__global__ void k_res_eoff(const int32_t *vtx_off, int32_t n, const int32_t *rowptr, const int32_t *emp,
                           int32_t *eoff) {
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; g <= n; g += gridDim.x * blockDim.x) {
        const int32_t v = vtx_off[g];
        eoff[g] = rowptr[v] + emp[v];
    }
}

// A warp per vertex v: its row goes to stream position rowptr[v] + emp[v] (emp = empty rows
// before v) as sources relative to the graph's compact numbering, or, when it has no in-edge,
// as one edge from the graph's zero slot; the row's first edge gets a head bit.
__global__ void k_res_stream(const int32_t *rowptr, const int32_t *colidx, const int32_t *cpos, const int32_t *gid,
                             const int32_t *vtx_off, const int32_t *emp, int32_t V, uint16_t *src16,
                             uint32_t *heads32) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < V; v += warps) {
        const int32_t s = rowptr[v], e = rowptr[v + 1], p = s + emp[v];
        const int32_t g = gid[v];
        const int32_t cg = cpos[vtx_off[g]];
        if (lane == 0) atomicOr(heads32 + (p >> 5), 1u << (p & 31));
        if (s == e) {
            if (lane == 0) src16[p] = (uint16_t)(cpos[vtx_off[g + 1]] - cg);
        } else {
            for (int32_t i = s + lane; i < e; i += 32) src16[p + (i - s)] = (uint16_t)(cpos[colidx[i]] - cg);
        }
    }
}

// heads of every 512-edge chunk (16 words)
__global__ void k_res_chunk_heads(const uint32_t *heads32, int64_t chunks, int32_t *cnt) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < chunks; c += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) k += __popc(heads32[16 * c + i]);
        cnt[c] = k;
    }
}

// Builds (once) what the resident variant reads; sets m->res_ok when every graph's
// non-dangling vertices fit one CTA's shared memory and 16-bit indices.
static int build_resident(tc_multigraph *m, cudaStream_t s) {
    if (m->res_built) return TC_OK;
    const int32_t V = m->g->V, n = m->n;
    const int64_t E = m->g->E;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    DevBuf flag, sizes, edges;
    TC_TRY(flag.alloc((size_t)(V > 0 ? V : 1) * 4));
    TC_TRY(m->cpos.alloc(((size_t)V + 1) * 4));
    TC_TRY(sizes.alloc((size_t)n * 4));
    TC_TRY(edges.alloc((size_t)n * 4));
    k_multi_nondangling<<<caps.sms * 8, 256, 0, s>>>(m->g->inv_outdeg.as<float>(), V, flag.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32(flag.as<int32_t>(), V, m->cpos.as<int32_t>(), s));
    k_multi_cpos_end<<<1, 1, 0, s>>>(m->cpos.as<int32_t>(), flag.as<int32_t>(), V);
    TC_LAUNCH_CHECK();
    k_multi_graph_sizes<<<(n + 255) / 256, 256, 0, s>>>(m->vtx_off.as<int32_t>(), n, m->cpos.as<int32_t>(),
                                                       m->g->in_rowptr.as<int32_t>(), sizes.as<int32_t>(),
                                                       edges.as<int32_t>());
    TC_LAUNCH_CHECK();
    int32_t *hs = new (std::nothrow) int32_t[2 * (size_t)n];
    if (!hs) return fail(TC_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(hs, sizes.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs + n, edges.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete[] hs;
        return fail(TC_ERR_CUDA, "build_resident: %s", cudaGetErrorString(e));
    }
    int32_t mx = 0;
    for (int32_t g = 0; g < n; ++g) mx = hs[g] > mx ? hs[g] : mx;
    std::vector<int32_t> ord((size_t)n);
    for (int32_t g = 0; g < n; ++g) ord[g] = g;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return hs[n + x] > hs[n + y]; });
    delete[] hs;
    m->res_max = mx;
    // shared memory holds the contributions and the zero slot; sources are 16-bit
    m->res_ok = mx + 1 <= 65536 && (size_t)(mx + 1) * 4 + 1024 <= (size_t)caps.max_smem_optin;
    if (m->res_ok) {
        DevBuf emp;
        TC_TRY(emp.alloc(((size_t)V + 1) * 4));
        TC_TRY(m->eoff.alloc(((size_t)n + 1) * 4));
        if (V > 0) {
            k_res_empty<<<caps.sms * 8, 256, 0, s>>>(m->g->in_rowptr.as<int32_t>(), V, flag.as<int32_t>());
            TC_LAUNCH_CHECK();
            TC_TRY(scan_i32(flag.as<int32_t>(), V, emp.as<int32_t>(), s));
        }
        k_multi_cpos_end<<<1, 1, 0, s>>>(emp.as<int32_t>(), flag.as<int32_t>(), V);
        TC_LAUNCH_CHECK();
        k_res_eoff<<<(n + 256) / 256, 256, 0, s>>>(m->vtx_off.as<int32_t>(), n, m->g->in_rowptr.as<int32_t>(),
                                                   emp.as<int32_t>(), m->eoff.as<int32_t>());
        TC_LAUNCH_CHECK();
        int32_t empties = 0;
        TC_CUDA(cudaMemcpyAsync(&empties, emp.as<int32_t>() + V, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        const int64_t Ep = E + empties;
        if (Ep + 2 * MR_CHUNK > INT32_MAX) {
            m->res_ok = false;
        } else {
            // whole 512-edge chunks plus one: a warp reads its last chunk (and the head words of
            // its first) in full, past the final edge
            const int64_t chunks = Ep / MR_CHUNK + 2;
            TC_TRY(m->order.alloc((size_t)n * 4));
            TC_TRY(m->src16.alloc((size_t)chunks * MR_CHUNK * 2));
            TC_TRY(m->heads.alloc((size_t)chunks * (MR_CHUNK / 8)));
            TC_TRY(m->hpre.alloc((size_t)chunks * 4));
            TC_TRY(m->scratch.alloc((size_t)(V > 0 ? V : 1) * 4));
            DevBuf cnt;
            TC_TRY(cnt.alloc((size_t)chunks * 4));
            TC_CUDA(cudaMemcpyAsync(m->order.p, ord.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
            TC_CUDA(cudaMemsetAsync(m->src16.p, 0, (size_t)chunks * MR_CHUNK * 2, s));
            TC_CUDA(cudaMemsetAsync(m->heads.p, 0, (size_t)chunks * (MR_CHUNK / 8), s));
            if (V > 0) {
                k_res_stream<<<caps.sms * 8, 256, 0, s>>>(m->g->in_rowptr.as<int32_t>(), m->g->in_colidx.as<int32_t>(),
                                                          m->cpos.as<int32_t>(), m->gid.as<int32_t>(),
                                                          m->vtx_off.as<int32_t>(), emp.as<int32_t>(), V,
                                                          m->src16.as<uint16_t>(), m->heads.as<uint32_t>());
                TC_LAUNCH_CHECK();
            }
            k_res_chunk_heads<<<(int)((chunks + 255) / 256), 256, 0, s>>>(m->heads.as<uint32_t>(), chunks,
                                                                          cnt.as<int32_t>());
            TC_LAUNCH_CHECK();
            TC_TRY(scan_i32(cnt.as<int32_t>(), chunks, m->hpre.as<int32_t>(), s));
            TC_CUDA(cudaStreamSynchronize(s));
        }
    }
    m->res_built = true;
    return TC_OK;
}

static size_t res_smem_bytes(const tc_multigraph *m) {
    return (size_t)((m->res_max + 1 + 3) & ~3) * 4;
}

typedef void (*MultiKernel)(MultiArgs);
static MultiKernel multi_kernel(int lanes) {
    switch (lanes) {
        case 1: return k_multi_pagerank<1>;
        case 4: return k_multi_pagerank<4>;
        case 8: return k_multi_pagerank<8>;
        case 32: return k_multi_pagerank<32>;
        default: return k_multi_pagerank<0>;
    }
}

static int multi_grid(int lanes, int ctas_per_sm, int *grid, size_t res_smem = 0) {
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    int per_sm = 0;
    if (lanes == TC_MULTI_RESIDENT) {
        TC_CUDA(cudaFuncSetAttribute(k_multi_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)res_smem));
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_resident, MR_THREADS, res_smem));
    } else {
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)multi_kernel(lanes), MU_THREADS, 0));
    }
    if (per_sm < 1) return fail(TC_ERR_CUDA, "k_multi_pagerank cannot be resident");
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    *grid = caps.sms * per_sm;
    return TC_OK;
}

// Clears the barrier words and the dangling accumulators, then launches the persistent kernel.
static int launch_multi(tc_multigraph *m, const MultiArgs &a, int lanes, int grid, cudaStream_t s) {
    TC_CUDA(cudaMemsetAsync(m->sync.p, 0, 16, s));
    if (lanes == TC_MULTI_RESIDENT) {
        ResArgs r;
        r.src16 = m->src16.as<uint16_t>();
        r.heads = m->heads.as<uint16_t>();
        r.hpre = m->hpre.as<int32_t>();
        r.eoff = m->eoff.as<int32_t>();
        r.cpos = m->cpos.as<int32_t>();
        r.vtx_off = m->vtx_off.as<int32_t>();
        r.order = m->order.as<int32_t>();
        r.inv_outdeg = a.inv_outdeg;
        r.n = a.n;
        r.iters = a.iters;
        r.drop = a.drop;
        r.damping = a.damping;
        r.sums = m->scratch.as<float>();
        r.rank = a.rank;
        r.next = m->sync.as<unsigned>() + 3;
        k_multi_resident<<<grid, MR_THREADS, res_smem_bytes(m), s>>>(r);
        TC_LAUNCH_CHECK();
        return TC_OK;
    }
    TC_CUDA(cudaMemsetAsync(m->dacc.p, 0, (size_t)3 * m->n * 8, s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(MU_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TC_CUDA(cudaLaunchKernelEx(&cfg, multi_kernel(lanes), a));
    return TC_OK;
}

static MultiArgs make_args(tc_multigraph *m, const tc_pr_params *pp) {
    MultiArgs a;
    a.rowptr = m->g->in_rowptr.as<int32_t>();
    a.colidx = m->g->in_colidx.as<int32_t>();
    a.gid = m->gid.as<int32_t>();
    a.inv_outdeg = m->g->inv_outdeg.as<float>();
    a.invVg = m->invVg.as<float>();
    a.V = m->g->V;
    a.n = m->n;
    a.iters = pp->iters;
    a.drop = pp->dangling == TC_DANGLING_DROP;
    a.damping = pp->damping;
    a.Vp = ((int64_t)a.V + 63) / 64 * 64;
    a.contrib = m->contrib.as<float>();
    a.rank = m->rank.as<float>();
    a.dacc = m->dacc.as<unsigned long long>();
    a.bar = m->sync.as<unsigned>();
    a.err = reinterpret_cast<int *>(m->sync.as<unsigned>() + 2);
    return a;
}

// One run: clear the barrier/error words, then the persistent kernel (through the cached
// CUDA graph when use_graph).
static int run_multi(tc_multigraph *m, const tc_pr_params *pp, int lanes, int ctas_per_sm, bool use_graph,
                     cudaStream_t s) {
    int grid = 0;
    if (lanes == TC_MULTI_RESIDENT) {
        TC_TRY(build_resident(m, s));
        if (!m->res_ok)
            return fail(TC_ERR_UNSUPPORTED, "TC_MULTI_RESIDENT: a graph has %d non-dangling vertices, more than one "
                        "CTA's shared memory holds", m->res_max);
    }
    TC_TRY(multi_grid(lanes, ctas_per_sm, &grid, res_smem_bytes(m)));
    const MultiArgs a = make_args(m, pp);
    if (!use_graph) return launch_multi(m, a, lanes, grid, s);
    const bool same = m->exec && m->cached_damping == pp->damping && m->cached_iters == pp->iters &&
                      m->cached_drop == a.drop && m->cached_lanes == lanes && m->cached_ctas == grid;
    if (!same) {
        if (m->exec) {
            cudaGraphExecDestroy(m->exec);
            m->exec = nullptr;
        }
        cudaStream_t cs;
        TC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int st = TC_OK;
        if (e == cudaSuccess) {
            st = launch_multi(m, a, lanes, grid, cs);
            cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && st == TC_OK) e = cudaGraphInstantiate(&m->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (st != TC_OK) return st;
        if (e != cudaSuccess) {
            m->exec = nullptr;
            return fail(TC_ERR_CUDA, "capturing the persistent launch failed: %s", cudaGetErrorString(e));
        }
        m->cached_damping = pp->damping;
        m->cached_iters = pp->iters;
        m->cached_drop = a.drop;
        m->cached_lanes = lanes;
        m->cached_ctas = grid;
    }
    TC_CUDA(cudaGraphLaunch(m->exec, s));
    return TC_OK;
}

static int timed_run(tc_multigraph *m, const tc_pr_params *pp, int lanes, cudaStream_t s, float *ms) {
    cudaEvent_t ev[2];
    TC_CUDA(cudaEventCreate(&ev[0]));
    TC_CUDA(cudaEventCreate(&ev[1]));
    TC_CUDA(cudaEventRecord(ev[0], s));
    int st = run_multi(m, pp, lanes, 0, false, s);
    cudaEventRecord(ev[1], s);
    cudaEventSynchronize(ev[1]);
    cudaEventElapsedTime(ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    return st;
}

}  // namespace tc

extern "C" int tc_multigraph_load(int32_t num_graphs, const int32_t *vtx_off, int32_t V, int64_t E,
                                  const int32_t *rowptr, const int32_t *colidx, int mem, void *stream,
                                  tc_multigraph **out) {
    using namespace tc;
    if (!out) return fail(TC_ERR_INVALID_ARG, "tc_multigraph_load: out is NULL");
    *out = nullptr;
    if (num_graphs < 1 || !vtx_off) return fail(TC_ERR_INVALID_ARG, "tc_multigraph_load: no graphs");
    if (vtx_off[0] != 0 || vtx_off[num_graphs] != V)
        return fail(TC_ERR_INVALID_ARG, "tc_multigraph_load: vtx_off must run from 0 to V");
    for (int32_t g = 0; g < num_graphs; ++g)
        if (vtx_off[g + 1] < vtx_off[g]) return fail(TC_ERR_INVALID_ARG, "tc_multigraph_load: vtx_off not monotone");
    cudaStream_t s = (cudaStream_t)stream;
    tc_graph *g = nullptr;
    TC_TRY(tc_graph_load_csr(V, E, rowptr, colidx, mem, stream, &g));
    tc_multigraph *m = new (std::nothrow) tc_multigraph();
    if (!m) {
        tc_graph_free(g);
        return fail(TC_ERR_OOM, "host allocation failed");
    }
    m->g = g;
    m->n = num_graphs;
    int st = m->vtx_off.alloc(((size_t)num_graphs + 1) * 4);
    if (st == TC_OK) st = m->gid.alloc((size_t)(V > 0 ? V : 1) * 4);
    if (st == TC_OK) st = m->invVg.alloc((size_t)num_graphs * 4);
    const int64_t Vp = ((int64_t)V + 63) / 64 * 64;
    if (st == TC_OK) st = m->rank.alloc((size_t)(V > 0 ? V : 1) * 4);
    if (st == TC_OK) st = m->contrib.alloc((size_t)(2 * Vp + 64) * 4);
    if (st == TC_OK) st = m->dacc.alloc((size_t)3 * num_graphs * 8);
    if (st == TC_OK) st = m->sync.alloc(64);
    if (st != TC_OK) {
        delete m;
        return st;
    }
    cudaError_t e = cudaMemcpyAsync(m->vtx_off.p, vtx_off, ((size_t)num_graphs + 1) * 4, cudaMemcpyHostToDevice, s);
    DeviceCaps caps;
    if (e == cudaSuccess && (st = device_caps(&caps)) == TC_OK) {
        k_multi_gid<<<caps.sms * 8, 256, 0, s>>>(m->vtx_off.as<int32_t>(), num_graphs, V, m->gid.as<int32_t>(),
                                                 m->invVg.as<float>());
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemsetAsync(m->sync.p, 0, 64, s);
        if (e == cudaSuccess && V > 0) {
            k_multi_check<<<caps.sms * 8, 256, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(),
                                                       m->gid.as<int32_t>(), V, reinterpret_cast<int *>(m->sync.p));
            e = cudaGetLastError();
        }
        int bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, m->sync.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && bad) st = fail(TC_ERR_INVALID_GRAPH, "tc_multigraph_load: an edge joins two graphs");
        if (e == cudaSuccess) e = cudaMemsetAsync(m->sync.p, 0, 64, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) st = fail(TC_ERR_CUDA, "tc_multigraph_load: %s", cudaGetErrorString(e));
    if (st != TC_OK) {
        delete m;
        return st;
    }
    *out = m;
    return TC_OK;
}

extern "C" void tc_multigraph_free(tc_multigraph *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    delete m;
}

extern "C" int tc_multi_autotune(tc_multigraph *m, const tc_pr_params *params, int32_t *best_lanes, float *times_ms,
                                 void *stream) {
    using namespace tc;
    if (!m || !params) return fail(TC_ERR_INVALID_ARG, "tc_multi_autotune: null argument");
    if (m->g->V == 0) return fail(TC_ERR_INVALID_ARG, "tc_multi_autotune: empty batch");
    cudaStream_t s = (cudaStream_t)stream;
    float best = 3.4e38f;
    int best_l = -1;
    TC_TRY(build_resident(m, s));
    for (int k = 0; k < MU_NVARIANTS; ++k) {
        float ms = 0, ms2 = 0;
        if (kLanes[k] == TC_MULTI_RESIDENT && !m->res_ok) {
            if (times_ms) times_ms[k] = -1.0f;
            continue;
        }
        TC_TRY(timed_run(m, params, kLanes[k], s, &ms));   // warm-up
        TC_TRY(timed_run(m, params, kLanes[k], s, &ms2));
        if (times_ms) times_ms[k] = ms2;
        if (ms2 < best) {
            best = ms2;
            best_l = kLanes[k];
        }
    }
    int err = 0;
    TC_CUDA(cudaMemcpyAsync(&err, m->sync.as<unsigned>() + 2, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (err) return fail(TC_ERR_TIMEOUT, "tc_multi_autotune: a grid barrier gave up");
    m->tuned_lanes = best_l;
    if (best_lanes) *best_lanes = best_l;
    return TC_OK;
}

extern "C" int tc_pagerank_multi(const tc_multigraph *cm, const tc_pr_params *params, const tc_multi_params *mp,
                                 float *ranks_out, tc_pr_stats *stats, void *stream) {
    using namespace tc;
    tc_multigraph *m = const_cast<tc_multigraph *>(cm);
    if (!m || !params || !ranks_out) return fail(TC_ERR_INVALID_ARG, "tc_pagerank_multi: null argument");
    if (!(params->damping >= 0.0f && params->damping <= 1.0f) || params->iters < 0)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_multi: damping outside [0,1] or iters < 0");
    if (params->dangling != TC_DANGLING_REDISTRIBUTE && params->dangling != TC_DANGLING_DROP)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_multi: bad dangling mode");
    if (params->out_mem != TC_MEM_HOST && params->out_mem != TC_MEM_DEVICE)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_multi: bad out_mem");
    if (params->init) return fail(TC_ERR_UNSUPPORTED, "tc_pagerank_multi: init ranks are not supported");
    int lanes = mp ? mp->lanes_per_vertex : 0;
    if (lanes == 0) lanes = m->tuned_lanes ? m->tuned_lanes : -1;
    if (lanes != -1 && lanes != 1 && lanes != 4 && lanes != 8 && lanes != 32 && lanes != TC_MULTI_RESIDENT)
        return fail(TC_ERR_INVALID_ARG,
                    "tc_pagerank_multi: lanes_per_vertex must be 0, -1, 1, 4, 8, 32 or TC_MULTI_RESIDENT");
    const bool use_graph = mp ? mp->use_graph != 0 : true;
    const int ctas = mp ? mp->ctas_per_sm : 0;
    cudaStream_t s = (cudaStream_t)stream;
    if (m->g->V == 0) return TC_OK;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (params->profile) {
        TC_CUDA(cudaEventCreate(&ev[0]));
        TC_CUDA(cudaEventCreate(&ev[1]));
        TC_CUDA(cudaEventRecord(ev[0], s));
    }
    TC_TRY(run_multi(m, params, lanes, ctas, use_graph && ctas == 0, s));
    float ms = 0;
    if (params->profile) {
        TC_CUDA(cudaEventRecord(ev[1], s));
        TC_CUDA(cudaEventSynchronize(ev[1]));
        TC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    const cudaMemcpyKind kind = params->out_mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TC_CUDA(cudaMemcpyAsync(ranks_out, m->rank.p, (size_t)m->g->V * 4, kind, s));
    if (stats || params->out_mem == TC_MEM_HOST) {
        int err = 0;
        TC_CUDA(cudaMemcpyAsync(&err, m->sync.as<unsigned>() + 2, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        if (err) return fail(TC_ERR_TIMEOUT, "tc_pagerank_multi: a grid barrier gave up");
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iters = params->iters;
        stats->launches = 1;
        stats->ms_total = ms;
        stats->ms_gather = ms;
    }
    return TC_OK;
}
