// Personalised PageRank for a batch of sources (one column per source), pull direction.
// Column j follows Alg. 1 with the teleport term (1-d) and the dangling mass of column j sent
// to its own source s_j, starting from e_{s_j}:
//   R'[v,j] = d * sum_{u->v} R[u,j] / out_degree[u] + [v == s_j] ((1-d) + d * D_j),
//   D_j     = sum over dangling u of R[u,j].
// The batch is an FP32 [V x n] row-major matrix; one warp gathers whole rows of the
// contribution matrix (n floats, float4 per lane), so every in-edge costs one coalesced row
// read.  Per-column dangling sums are accumulated in 64-bit fixed point (deterministic).
//
// Without a partition the batch runs as ONE persistent cooperative launch for all iterations
// (two grid barriers per iteration), captured once in a CUDA graph and replayed.  It works in the
// vertex numbering by out-degree: the sources with the most out-edges come first, so their rows
// (which most in-edges read) are one contiguous range, and the two contribution matrices are
// interleaved row by row so that the hot rows of both form one range too.  That range - the
// paper's source block sized to the last-level cache (Sec. 3.1), here without partial sums - is
// kept in L2 by an access-policy window; an autotuner picks its size and the launch width.
#include <cooperative_groups.h>

#include "tc_common_dev.cuh"

namespace tc {

// Compensated (Kahan) addition of y into (sum, c).  A column of a personalised batch often sums
// thousands of nearly equal small contributions next to one large one; plain sequential FP32
// addition then rounds the same way every time and drifts.
__device__ __forceinline__ void kahan_add(float &sum, float &c, float y) {
    const float yc = y - c;
    const float t = sum + yc;
    c = (t - sum) - yc;
    sum = t;
}

__device__ __forceinline__ void kahan_add4(float4 &sum, float4 &c, float4 y) {
    kahan_add(sum.x, c.x, y.x);
    kahan_add(sum.y, c.y, y.y);
    kahan_add(sum.z, c.z, y.z);
    kahan_add(sum.w, c.w, y.w);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

// L2 eviction priorities for the persistent batch (createpolicy, per access): the contribution
// rows of the `hot` sources with the most out-edges - those most in-edges read - are loaded and
// stored evict-last; the other rows and the in-edge lists (read once per iteration) are
// evict-first.  With hot = 0 every such access is evict-normal.
struct PprHints {
    uint64_t last, cold;
    int32_t hot;
};

__device__ __forceinline__ uint64_t l2_policy_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_policy_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ PprHints ppr_hints(int32_t hot) {
    PprHints h;
    h.last = l2_policy_last();
    h.cold = hot > 0 ? l2_policy_first() : l2_policy_normal();
    h.hot = hot;
    return h;
}
// A float4 from L2 (not L1: the data were written in this launch by other SMs) with a policy.
__device__ __forceinline__ float4 ld_f4_hint(const float4 *p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_i32_hint(const int32_t *p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_f4_hint(float4 *p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}

constexpr int PPR_THREADS = 256;
constexpr int PPR_DEFAULT_TILE = 32;  // columns per tile of the persistent batch until it is tuned
constexpr int PPR_WARPS = PPR_THREADS / 32;
constexpr double PPR_FX = 2305843009213693952.0;  // 2^61: every column has L1 mass <= 1

// A dangling row's value in the fixed point of the per-column sums.  Rows reach warps in the
// order a work queue hands them out, so the sums are integers: exact, in any order.
// r = m * 2^(e - 150) (m the 24-bit significand, e the biased exponent) for 0 <= r <= 1, so
// r * 2^61 = m * 2^(e - 89): a shift of m, rounded half up where it drops bits.  Integer
// operations only: 64-bit float-to-integer conversions run on the FP64 unit, which this GPU
// has little of.
__device__ __forceinline__ unsigned long long ppr_fx(float r) {
    const uint32_t b = __float_as_uint(r) & 0x7fffffffu;
    const int e = (int)(b >> 23);
    const unsigned long long m = (b & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = (e ? e : 1) - 89;
    if (sh >= 0) return m << sh;
    if (sh <= -25) return 0ull;  // below 2^-62: rounds to 0 (m < 2^24)
    return (m + (1ull << (-sh - 1))) >> (-sh);
}

// Rows with more than PPR_PIECE in-edges are cut into pieces of PPR_PIECE edges, each summed by
// its own warp into a partial row (k_ppr_piece), and finished by k_ppr_fix, which adds the
// pieces of a row in order: a hub no longer serialises a whole iteration on one warp.
constexpr int PPR_PIECE = 2048;

// Sum of the contribution rows of in-edges [s, e) (row u at C + u * rs4 float4), float4 per
// lane.  The rows were written earlier in the same launch by other SMs, so they are read from
// L2 (ld.global.cg): an SM's L1 may still hold the lines of the same buffer from two iterations
// before, and a grid barrier does not clear it.
template <int NV4>
__device__ __forceinline__ void ppr_row_sum(const int32_t *__restrict__ colidx, int32_t s, int32_t e,
                                            const float4 *C, int64_t rs4, int lane, float4 *acc, const PprHints &h) {
    constexpr int U = NV4 <= 2 ? 4 : 2;  // rows in flight (a power of two)
    float4 comp[NV4];
#pragma unroll
    for (int q = 0; q < NV4; ++q) comp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int32_t i = s;
    for (; i + U - 1 < e; i += U) {
        int64_t u[U];
#pragma unroll
        for (int k2 = 0; k2 < U; ++k2) u[k2] = __ldg(colidx + i + k2);
        float4 x[U][NV4];
#pragma unroll
        for (int k2 = 0; k2 < U; ++k2)
#pragma unroll
            for (int q = 0; q < NV4; ++q) x[k2][q] = ld_f4_hint(C + u[k2] * rs4 + 32 * q + lane, u[k2] < h.hot ? h.last : h.cold);
#pragma unroll
        for (int q = 0; q < NV4; ++q) {  // tree sum of the group, then one compensated add
            float4 gsum = add4(x[0][q], x[1][q]);
            if (U == 4) gsum = add4(gsum, add4(x[2][q], x[3][q]));
            kahan_add4(acc[q], comp[q], gsum);
        }
    }
    for (; i < e; ++i) {
        const int64_t u0 = __ldg(colidx + i);
#pragma unroll
        for (int q = 0; q < NV4; ++q)
            kahan_add4(acc[q], comp[q], ld_f4_hint(C + u0 * rs4 + 32 * q + lane, u0 < h.hot ? h.last : h.cold));
    }
}

// Grid-wide barrier with a bounded spin (about a second); on a timeout it records code 5.
__device__ __forceinline__ bool ppr_grid_barrier(unsigned *bar, int *err) {
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
                    atomicCAS(err, 0, 5);
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

// Queue items after the pieces are built from runs of consecutive rows whose cost (light
// in-edges plus PPR_ROW_COST per row, for the row's update and its store) is about PPR_SUB_COST:
// a whole-row item walks PPR_SUB_PER_ITEM runs as one stream, a tiled item gives one run to
// each lane group of the warp.
constexpr int PPR_SUB_COST = 512;
constexpr int PPR_SUB_PER_ITEM = 4;
constexpr int PPR_ROW_COST = 8;

struct PprArgs {
    const int32_t *rowptr, *colidx;      // G^T in the numbering by out-degree (read by the pieces)
    const int32_t *rowptr_l, *colidx_l;  // the same rows without the in-edges of the long rows
    const int32_t *chunk_row;            // [nsub + 1] first row of every run
    int32_t nsub;
    int32_t V, n, iters, np;
    float *CC;                           // interleaved: row u of matrix b at CC + (2 u + b) * NP floats
    const int32_t *srcc;                 // [NP] source (new ID) of every column, -1 for padding
    unsigned long long *D;               // [3][NP] fixed-point dangling sums (current, next, to clear)
    const float *inv_outdeg;             // new order
    float damping;
    float *R_out;                        // [V x n] by the caller's IDs, written in the last iteration
    const int32_t *perm;                 // new ID -> caller's ID
    const uint8_t *is_src;               // new IDs: 1 where some column teleports
    const uint8_t *is_long;              // new IDs: 1 for the rows cut into pieces
    const int32_t *hub_rows, *hub_piece0;
    const int2 *pieces;
    int32_t nhubs, npieces;
    int32_t hot;                         // rows kept in L2 with evict-last accesses
    float *Ppc;                          // [npieces][NP] partial rows of the long rows
    unsigned *hub_count;                 // [nhubs] pieces of the row finished in this iteration
    unsigned *sync;                      // [0] barrier count, [1] generation, [2] error, [4..6] queue heads
};

// Row v's new values from its in-edge sum acc (Alg. 1 with the teleport of the columns whose
// source is v): the next contribution row, the dangling sums of the warp's columns and, in the
// last iteration, the output row.
template <int NV4>
__device__ __forceinline__ void ppr_finish(const PprArgs &a, int64_t v, const float4 *acc, float4 *Cn, bool last,
                                           const int32_t *ssrc, const float *stele, unsigned long long *dsw, int lane,
                                           const PprHints &h) {
    constexpr int64_t RS4 = 64 * NV4;  // float4 from one row of a matrix to the next
    const float inv = __ldg(a.inv_outdeg + v);
    const bool vsrc = __ldg(a.is_src + v) != 0;  // the same byte for the whole warp
    const int64_t ro = last && a.R_out ? (int64_t)__ldg(a.perm + v) * a.n : -1;
#pragma unroll
    for (int q = 0; q < NV4; ++q) {
        float r[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = 128 * q + 4 * lane + c;
            r[c] = a.damping * r[c] + ((vsrc && ssrc[j] == (int32_t)v) ? stele[j] : 0.0f);
            if (inv == 0.0f) dsw[j] += ppr_fx(r[c]);  // lane-owned columns: no race
        }
        st_f4_hint(Cn + v * RS4 + 32 * q + lane, make_float4(r[0] * inv, r[1] * inv, r[2] * inv, r[3] * inv),
                   v < h.hot ? h.last : h.cold);
        if (ro >= 0) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = 128 * q + 4 * lane + c;
                if (j < a.n) __stcs(a.R_out + ro + j, r[c]);
            }
        }
    }
}

// One persistent cooperative launch runs every iteration.  In each, warps draw items from a
// queue: first the pieces of the long rows (the last piece of a row to finish adds the row's
// pieces in order and updates it), then runs of consecutive light rows, walked as one edge stream
// with U in-edges in flight whatever the row boundaries, so that rows with a few in-edges do not
// leave the warp waiting on one load at a time.  A grid barrier ends the iteration.
// Every access to the contribution matrices and the pieces goes through L2 (see ppr_row_sum).
// Every row's sum has a fixed order (fixed runs and groups), whatever the launch width.
template <int NV4>
__global__ void __launch_bounds__(PPR_THREADS, NV4 == 1 ? 4 : (NV4 == 2 ? 3 : (NV4 == 4 ? 2 : 1))) k_ppr_persist(PprArgs a) {
    constexpr int NP = 128 * NV4;
    constexpr int64_t RS4 = NP / 2;  // a row of one matrix is NP/4 float4; rows are two of those apart
    constexpr int U = NV4 <= 2 ? 4 : 2;
    // per-column constants live in shared memory (registers go to rows in flight): the source
    // vertex and teleport term of each column, and each warp's dangling sums
    extern __shared__ unsigned long long dsh_dyn[];  // [PPR_WARPS][NP]
    __shared__ int32_t ssrc[NP];
    __shared__ float stele[NP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned nitems = (unsigned)a.npieces + (unsigned)((a.nsub + PPR_SUB_PER_ITEM - 1) / PPR_SUB_PER_ITEM);
    unsigned *queue = a.sync + 4;
    int *err = reinterpret_cast<int *>(a.sync + 2);
    unsigned long long *dsw = dsh_dyn + warp * NP;
    const PprHints h = ppr_hints(a.hot);
    for (int j = threadIdx.x; j < NP; j += PPR_THREADS) ssrc[j] = a.srcc[j];
    for (int it = 0; it < a.iters; ++it) {
        const bool last = it == a.iters - 1;
        const int cur = it & 1;
        const float4 *Cc = reinterpret_cast<const float4 *>(a.CC) + cur * (NP / 4);
        float4 *Cn = reinterpret_cast<float4 *>(a.CC) + (cur ^ 1) * (NP / 4);
        const unsigned long long *Dc = a.D + (it % 3) * NP;
        unsigned long long *Dn = a.D + ((it + 1) % 3) * NP, *Dz = a.D + ((it + 2) % 3) * NP;
        if (blockIdx.x == 0) {  // the buffers of iteration it + 2 were last used in iteration it - 1
            for (int j = threadIdx.x; j < NP; j += PPR_THREADS) Dz[j] = 0ull;
            if (threadIdx.x == 0) queue[(it + 2) % 3] = 0u;
        }
        for (int j = threadIdx.x; j < NP; j += PPR_THREADS)
            stele[j] = (1.0f - a.damping) + a.damping * (float)((double)__ldcg(Dc + j) / PPR_FX);
        for (int j = lane; j < NP; j += 32) dsw[j] = 0ull;
        __syncthreads();
        while (true) {
            unsigned item = 0;
            if (lane == 0) item = atomicAdd(queue + it % 3, 1u);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item >= nitems) break;
            float4 acc[NV4];
#pragma unroll
            for (int q = 0; q < NV4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (item < (unsigned)a.npieces) {
                const int2 pc = a.pieces[item];
                const int32_t e = min(pc.y + PPR_PIECE, __ldg(a.rowptr + pc.x + 1));
                ppr_row_sum<NV4>(a.colidx, pc.y, e, Cc, RS4, lane, acc, h);
                float4 *dst = reinterpret_cast<float4 *>(a.Ppc) + (int64_t)item * (NP / 4);
#pragma unroll
                for (int q = 0; q < NV4; ++q) dst[32 * q + lane] = acc[q];
                int32_t lo = 0, hi = a.nhubs - 1;  // the row of this piece: last h with piece0[h] <= item
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(a.hub_piece0 + mid) <= (int32_t)item) lo = mid;
                    else hi = mid - 1;
                }
                const int32_t p0 = __ldg(a.hub_piece0 + lo), p1 = __ldg(a.hub_piece0 + lo + 1);
                __threadfence();
                __syncwarp();
                unsigned done = 0;
                if (lane == 0) done = atomicAdd(a.hub_count + lo, 1u);
                done = __shfl_sync(0xffffffffu, done, 0);
                if (done != (unsigned)(p1 - p0 - 1)) continue;  // another piece finishes the row
                __threadfence();
                if (lane == 0) a.hub_count[lo] = 0u;  // ready for the next iteration
#pragma unroll
                for (int q = 0; q < NV4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int32_t p = p0; p < p1; ++p)  // pieces in order
#pragma unroll
                    for (int q = 0; q < NV4; ++q)
                        acc[q] = add4(acc[q], __ldcg(reinterpret_cast<const float4 *>(a.Ppc) + (int64_t)p * (NP / 4) +
                                                     32 * q + lane));
                ppr_finish<NV4>(a, __ldg(a.hub_rows + lo), acc, Cn, last, ssrc, stele, dsw, lane, h);
                continue;
            }
            // a run of light rows [r, r1) as one stream of in-edges [i, e1)
            const int32_t c = (int32_t)(item - (unsigned)a.npieces) * PPR_SUB_PER_ITEM;
            int32_t r = __ldg(a.chunk_row + c);
            const int32_t r1 = __ldg(a.chunk_row + min(c + PPR_SUB_PER_ITEM, a.nsub));
            if (r >= r1) continue;
            int32_t i = __ldg(a.rowptr_l + r), rend = __ldg(a.rowptr_l + r + 1);
            const int32_t e1 = __ldg(a.rowptr_l + r1);
            float4 comp[NV4], x[U][NV4];
#pragma unroll
            for (int q = 0; q < NV4; ++q) comp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            int have = 0;  // in-edges i, i+1, ... already loaded into x[0], x[1], ...
            while (true) {
                if (rend <= i) {  // row r has all its in-edges
                    if (!__ldg(a.is_long + r)) ppr_finish<NV4>(a, r, acc, Cn, last, ssrc, stele, dsw, lane, h);
                    if (++r >= r1) break;
                    rend = __ldg(a.rowptr_l + r + 1);
#pragma unroll
                    for (int q = 0; q < NV4; ++q) acc[q] = comp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    continue;
                }
                if (have == 0) {
                    const int32_t cnt = min(U, e1 - i);
                    int64_t u[U];
#pragma unroll
                    for (int k2 = 0; k2 < U; ++k2) u[k2] = k2 < cnt ? ld_i32_hint(a.colidx_l + i + k2, h.cold) : -1;
#pragma unroll
                    for (int k2 = 0; k2 < U; ++k2)
#pragma unroll
                        for (int q = 0; q < NV4; ++q)
                            x[k2][q] = u[k2] >= 0 ? ld_f4_hint(Cc + u[k2] * RS4 + 32 * q + lane, u[k2] < h.hot ? h.last : h.cold)
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (i + cnt <= rend) {  // the group lies in row r: tree sum, one compensated add
#pragma unroll
                        for (int q = 0; q < NV4; ++q) {
                            float4 gsum = add4(x[0][q], x[1][q]);
#pragma unroll
                            for (int k2 = 2; k2 < U; k2 += 2) gsum = add4(gsum, add4(x[k2][q], x[k2 + 1][q]));
                            kahan_add4(acc[q], comp[q], gsum);
                        }
                        i += cnt;
                        continue;
                    }
                    have = cnt;
                }
#pragma unroll
                for (int q = 0; q < NV4; ++q) {  // one in-edge of row r, then shift the group
                    kahan_add4(acc[q], comp[q], x[0][q]);
#pragma unroll
                    for (int k2 = 0; k2 + 1 < U; ++k2) x[k2][q] = x[k2 + 1][q];
                }
                --have;
                ++i;
            }
        }
        // per-column dangling sums: warps -> shared -> one fixed-point atomic per column per CTA
        __syncthreads();
        for (int j = threadIdx.x; j < NP; j += PPR_THREADS) {
            unsigned long long t = 0ull;
#pragma unroll
            for (int w = 0; w < PPR_WARPS; ++w) t += dsh_dyn[w * NP + j];
            if (t != 0ull) atomicAdd(Dn + j, t);
        }
        if (!ppr_grid_barrier(a.sync, err)) return;
    }
}

// The tiled form of the persistent batch.  The columns run in tiles of TW = 128 / G: all the
// iterations of tile 0, then of tile 1, and so on (the columns of a batch are independent).
// Within a tile, a row of the contribution matrix is a TW * 4-byte segment, so the L2 keeps
// G times as many source rows as with whole rows: with TW = 32 a segment is one 128-byte line.
// A warp is G lane groups of 32 / G lanes, one float4 column group per lane; each group walks
// its own run of rows as one in-edge stream (U in-edges in flight), and all groups of the warp
// share a piece of a long row (in-edges strided by G, the group sums added in a fixed order).
template <int G>
__device__ __forceinline__ void ppr_finish_tile(const PprArgs &a, int64_t v, float4 acc, float4 *Cn, bool last,
                                                int c0, const int32_t *ssrc, const float *stele, unsigned long long *dsw,
                                                int gl,
                                                const PprHints &h) {
    const int64_t RS4 = a.np / 2;
    const float inv = __ldg(a.inv_outdeg + v);
    const bool vsrc = __ldg(a.is_src + v) != 0;
    float r[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = 4 * gl + c;
        r[c] = a.damping * r[c] + ((vsrc && ssrc[j] == (int32_t)v) ? stele[j] : 0.0f);
        if (inv == 0.0f) dsw[j] += ppr_fx(r[c]);  // lane-owned columns of the group: no race
    }
    st_f4_hint(Cn + v * RS4, make_float4(r[0] * inv, r[1] * inv, r[2] * inv, r[3] * inv), v < h.hot ? h.last : h.cold);
    if (last && a.R_out) {
        float *ro = a.R_out + (int64_t)__ldg(a.perm + v) * a.n + c0 + 4 * gl;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c0 + 4 * gl + c < a.n) __stcs(ro + c, r[c]);
    }
}

template <int G>
__global__ void __launch_bounds__(PPR_THREADS, 3) k_ppr_tiled(PprArgs a) {
    constexpr int L = 32 / G, TW = 128 / G, U = 8;
    __shared__ unsigned long long dsh[PPR_WARPS * G][TW];  // dangling sums of every lane group
    __shared__ int32_t ssrc[TW];
    __shared__ float stele[TW];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / L, gl = lane % L;
    const int NP = a.np;
    const int64_t RS4 = NP / 2;  // float4 from one row of a matrix to the next
    const int ntiles = (a.n + TW - 1) / TW;
    const unsigned nitems = (unsigned)a.npieces + (unsigned)((a.nsub + G - 1) / G);
    unsigned *queue = a.sync + 4;
    int *err = reinterpret_cast<int *>(a.sync + 2);
    unsigned long long *dsw = dsh[warp * G + grp];
    const PprHints h = ppr_hints(a.hot);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int step = 0;  // iterations over all tiles: selects the queue head
    for (int t = 0; t < ntiles; ++t) {
        const int c0 = t * TW;
        for (int it = 0; it < a.iters; ++it, ++step) {
            const bool last = it == a.iters - 1;
            const int cur = it & 1;
            // this lane's float4 of row 0 in both matrices; row u is u * RS4 float4 further
            const float4 *Cc = reinterpret_cast<const float4 *>(a.CC) + cur * (NP / 4) + c0 / 4 + gl;
            float4 *Cn = reinterpret_cast<float4 *>(a.CC) + (cur ^ 1) * (NP / 4) + c0 / 4 + gl;
            const unsigned long long *Dc = a.D + (it % 3) * NP + c0;
            unsigned long long *Dn = a.D + ((it + 1) % 3) * NP + c0, *Dz = a.D + ((it + 2) % 3) * NP + c0;
            if (blockIdx.x == 0) {  // buffers of iteration it + 2, last used in iteration it - 1
                for (int j = threadIdx.x; j < TW; j += PPR_THREADS) Dz[j] = 0ull;
                if (threadIdx.x == 0) queue[(step + 2) % 3] = 0u;
            }
            for (int j = threadIdx.x; j < TW; j += PPR_THREADS) {
                ssrc[j] = a.srcc[c0 + j];
                stele[j] = (1.0f - a.damping) + a.damping * (float)((double)__ldcg(Dc + j) / PPR_FX);
            }
            for (int j = gl; j < TW; j += L) dsw[j] = 0ull;
            __syncthreads();
            while (true) {
                unsigned item = 0;
                if (lane == 0) item = atomicAdd(queue + step % 3, 1u);
                item = __shfl_sync(0xffffffffu, item, 0);
                if (item >= nitems) break;
                if (item < (unsigned)a.npieces) {
                    // a piece of a long row: group g adds in-edges s + g, s + g + G, ...
                    const int2 pc = a.pieces[item];
                    const int32_t e = min(pc.y + PPR_PIECE, __ldg(a.rowptr + pc.x + 1));
                    float4 acc = zero4, comp = zero4;
                    for (int32_t i = pc.y + grp; i < e; i += G * U) {
                        float4 x[U];
#pragma unroll
                        for (int k = 0; k < U; ++k) {
                            const int32_t ie = i + G * k;
                            const int32_t u = ie < e ? ld_i32_hint(a.colidx + ie, h.cold) : -1;
                            x[k] = u >= 0 ? ld_f4_hint(Cc + (int64_t)u * RS4, u < h.hot ? h.last : h.cold) : zero4;
                        }
#pragma unroll
                        for (int k = U / 2; k >= 1; k /= 2)
#pragma unroll
                            for (int k2 = 0; k2 < k; ++k2) x[k2] = add4(x[k2], x[k2 + k]);
                        kahan_add4(acc, comp, x[0]);
                    }
#pragma unroll
                    for (int o = L; o < 32; o <<= 1) {  // the groups' sums, in a fixed order
                        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
                        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
                        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
                        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
                    }
                    float4 *Pp = reinterpret_cast<float4 *>(a.Ppc) + c0 / 4 + gl;
                    if (grp == 0) Pp[(int64_t)item * (NP / 4)] = acc;
                    int32_t lo = 0, hi = a.nhubs - 1;  // the row of this piece: last h with piece0[h] <= item
                    while (lo < hi) {
                        const int32_t mid = (lo + hi + 1) >> 1;
                        if (__ldg(a.hub_piece0 + mid) <= (int32_t)item) lo = mid;
                        else hi = mid - 1;
                    }
                    const int32_t p0 = __ldg(a.hub_piece0 + lo), p1 = __ldg(a.hub_piece0 + lo + 1);
                    __threadfence();
                    __syncwarp();
                    unsigned done = 0;
                    if (lane == 0) done = atomicAdd(a.hub_count + lo, 1u);
                    done = __shfl_sync(0xffffffffu, done, 0);
                    if (done != (unsigned)(p1 - p0 - 1)) continue;  // another piece finishes the row
                    __threadfence();
                    if (lane == 0) a.hub_count[lo] = 0u;  // ready for the next iteration
                    if (grp == 0) {
                        float4 sum = zero4;
                        for (int32_t p = p0; p < p1; ++p) sum = add4(sum, __ldcg(Pp + (int64_t)p * (NP / 4)));  // in order
                        ppr_finish_tile<G>(a, __ldg(a.hub_rows + lo), sum, Cn, last, c0, ssrc, stele, dsw, gl, h);
                    }
                    __syncwarp();
                    continue;
                }
                const int32_t sc = (int32_t)(item - (unsigned)a.npieces) * G + grp;
                if (sc < a.nsub) {  // the group's run of light rows [r, r1) as one in-edge stream
                    int32_t r = __ldg(a.chunk_row + sc);
                    const int32_t r1 = __ldg(a.chunk_row + sc + 1);
                    if (r < r1) {
                        int32_t i = __ldg(a.rowptr_l + r), rend = __ldg(a.rowptr_l + r + 1);
                        const int32_t e1 = __ldg(a.rowptr_l + r1);
                        float4 acc = zero4, comp = zero4, x[U];
                        int have = 0;  // in-edges i, i+1, ... already loaded into x[0], x[1], ...
                        while (true) {
                            if (rend <= i) {  // row r has all its in-edges
                                if (!__ldg(a.is_long + r))
                                    ppr_finish_tile<G>(a, r, acc, Cn, last, c0, ssrc, stele, dsw, gl, h);
                                if (++r >= r1) break;
                                rend = __ldg(a.rowptr_l + r + 1);
                                acc = comp = zero4;
                                continue;
                            }
                            if (have == 0) {
                                const int32_t cnt = min(U, e1 - i);
#pragma unroll
                                for (int k = 0; k < U; ++k) {
                                    const int32_t u = k < cnt ? ld_i32_hint(a.colidx_l + i + k, h.cold) : -1;
                                    x[k] = u >= 0 ? ld_f4_hint(Cc + (int64_t)u * RS4, u < h.hot ? h.last : h.cold) : zero4;
                                }
                                if (i + cnt <= rend) {  // the group lies in row r: tree sum, one compensated add
#pragma unroll
                                    for (int k = U / 2; k >= 1; k /= 2)
#pragma unroll
                                        for (int k2 = 0; k2 < k; ++k2) x[k2] = add4(x[k2], x[k2 + k]);
                                    kahan_add4(acc, comp, x[0]);
                                    i += cnt;
                                    continue;
                                }
                                have = cnt;
                            }
                            kahan_add4(acc, comp, x[0]);  // one in-edge of row r, then shift the group
#pragma unroll
                            for (int k = 0; k + 1 < U; ++k) x[k] = x[k + 1];
                            --have;
                            ++i;
                        }
                    }
                }
                __syncwarp();
            }
            // per-column dangling sums: groups -> one fixed-point atomic per column per CTA
            __syncthreads();
            for (int j = threadIdx.x; j < TW; j += PPR_THREADS) {
                unsigned long long tsum = 0ull;
#pragma unroll
                for (int w = 0; w < PPR_WARPS * G; ++w) tsum += dsh[w][j];
                if (tsum != 0ull) atomicAdd(Dn + j, tsum);
            }
            if (!ppr_grid_barrier(a.sync, err)) return;
        }
    }
}

// Light rows: deg_l[v] = in-degree of v unless v is cut into pieces (then 0); deg_l[V] = 0.
__global__ void k_ppr_light_deg(const int32_t *rowptr, int32_t V, int32_t *deg_l, uint8_t *is_long) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= V; v += (int64_t)gridDim.x * blockDim.x) {
        if (v == V) {
            deg_l[v] = 0;
            continue;
        }
        const int32_t d = rowptr[v + 1] - rowptr[v];
        const bool lg = d > PPR_PIECE;
        deg_l[v] = lg ? 0 : d;
        is_long[v] = lg ? 1 : 0;
    }
}

// colidx_l: the in-edges of the light rows, a warp per row.
__global__ void k_ppr_light_copy(const int32_t *rowptr, const int32_t *colidx, int32_t V, const int32_t *rowptr_l,
                                 int32_t *colidx_l) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < V; v += nw) {
        const int32_t s = rowptr_l[v], d = rowptr_l[v + 1] - s, so = rowptr[v];
        for (int32_t k = lane; k < d; k += 32) colidx_l[s + k] = colidx[so + k];
    }
}

// chunk_row[c] = first row r with rowptr_l[r] + PPR_ROW_COST * r >= c * target (c < nchunks), V at the end.
__global__ void k_ppr_chunks(const int32_t *rowptr_l, int32_t V, int64_t target, int32_t nchunks, int32_t *chunk_row) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c <= nchunks; c += (int64_t)gridDim.x * blockDim.x) {
        if (c == nchunks) {
            chunk_row[c] = V;
            continue;
        }
        const int64_t want = c * target;
        int32_t lo = 0, hi = V;
        while (lo < hi) {
            const int32_t mid = lo + (hi - lo) / 2;
            if ((int64_t)rowptr_l[mid] + (int64_t)PPR_ROW_COST * mid >= want) hi = mid;
            else lo = mid + 1;
        }
        chunk_row[c] = lo;
    }
}

// Columns in the numbering by out-degree: srcc[j] = inv[src_old[j]] (-1 past n), is_src marks
// them, D0[j] = the initial dangling mass of column j (1 when its source has no out-edges).
__global__ void k_ppr_columns(const int32_t *src_old, int32_t n, int32_t NP, const int32_t *inv,
                              const float *inv_outdeg, int32_t *srcc, uint8_t *is_src, unsigned long long *D0) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NP; j += gridDim.x * blockDim.x) {
        const int32_t u = j < n ? inv[src_old[j]] : -1;
        srcc[j] = u;
        D0[j] = 0ull;
        if (u < 0) continue;
        is_src[u] = 1;
        if (inv_outdeg[u] == 0.0f) D0[j] = (unsigned long long)PPR_FX;
    }
}

// R[s_j, j] = 1 (zero iterations: every column is its source's unit vector).
__global__ void k_ppr_unit(const int32_t *src, int32_t n, float *R) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        R[(int64_t)src[j] * n + j] = 1.0f;
}

// Matrix 0 of the interleaved pair: zero, then column j's source row holds 1 / out_degree.
__global__ void k_ppr_clear0(float4 *CC, int64_t V, int32_t NP) {
    const int64_t per = NP / 4;  // float4 per row of one matrix
    const int64_t total = V * per;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = t / per, c = t - u * per;
        CC[u * 2 * per + c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_ppr_seed(float *CC, int32_t NP, const int32_t *srcc, const float *inv_outdeg) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NP; j += gridDim.x * blockDim.x) {
        const int32_t u = srcc[j];
        if (u >= 0) CC[(int64_t)u * 2 * NP + j] = inv_outdeg[u];
    }
}

// C = e_{s_j} scaled by 1/out_degree(s_j); D0_j = [s_j dangling]; optional R_out = e_{s_j}.
__global__ void k_ppr_init(float *C, int32_t NP, const int32_t *src_of_col, const float *inv_outdeg,
                           unsigned long long *D0, float *R_out, int32_t n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NP; j += gridDim.x * blockDim.x) {
        const int32_t s = src_of_col[j];
        D0[j] = 0ull;
        if (s < 0) continue;
        const float inv = inv_outdeg[s];
        C[(int64_t)s * NP + j] = inv;
        if (inv == 0.0f) D0[j] = (unsigned long long)PPR_FX;
        if (R_out && j < n) R_out[(int64_t)s * n + j] = 1.0f;
    }
}

// ---------------------------------------------------------------------------------------------
// TOCAB form of the batch (Sec. 3.1 applied to a column tile): the n columns are processed in
// tiles of 32; for tile t the contribution matrix is read as 128-byte row segments C[u, 32t..]
// and the pull partition's source blocks are sized so that one block's segments stay in L2.
// Alg. 4 per block writes 32-wide partial rows; the merge of Fig. 5 (CTA per vertex range, the
// blocks added in block order - deterministic) applies the update for the tile's columns.
// ---------------------------------------------------------------------------------------------
constexpr int PT_THREADS = 256;
constexpr int PT_WARPS = PT_THREADS / 32;

constexpr int PT_PIECE = 1024;  // local rows above this many edges are cut into pieces

// Edges [s, e) of one row, tile t: 8 lanes (sub) each summing one float4 of the 32 columns.
__device__ __forceinline__ float4 tile_row_sum(const int32_t *__restrict__ colidx, int32_t s, int32_t e,
                                               const float4 *__restrict__ Ct, int64_t NP4) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
    int32_t i = s;
    for (; i + 3 < e; i += 4) {
        const int64_t u0 = __ldg(colidx + i), u1 = __ldg(colidx + i + 1), u2 = __ldg(colidx + i + 2),
                      u3 = __ldg(colidx + i + 3);
        const float4 x0 = __ldg(Ct + u0 * NP4), x1 = __ldg(Ct + u1 * NP4), x2 = __ldg(Ct + u2 * NP4),
                     x3 = __ldg(Ct + u3 * NP4);
        kahan_add4(a, c, add4(add4(x0, x1), add4(x2, x3)));
    }
    for (; i < e; ++i) kahan_add4(a, c, __ldg(Ct + (int64_t)__ldg(colidx + i) * NP4));
    return a;
}

// pieces of long local rows: 4 pieces per warp, 8 lanes each -> partial rows Ppc[piece][32]
__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_piece(const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const int2 *__restrict__ pieces, int32_t npieces,
                                                               const float *__restrict__ C, int32_t NP, int32_t t,
                                                               float *__restrict__ Ppc) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7, slot = lane >> 3;
    const int64_t nw = (int64_t)gridDim.x * PT_WARPS;
    const float4 *Ct = reinterpret_cast<const float4 *>(C + 32 * t) + sub;
    for (int64_t p0 = ((int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5)) * 4; p0 < npieces; p0 += nw * 4) {
        const int64_t p = p0 + slot;
        int32_t s = 0, e = 0;
        if (p < npieces) {
            const int2 pc = pieces[p];
            s = pc.y;
            e = min(pc.y + PT_PIECE, __ldg(rowptr + pc.x + 1));
        }
        const float4 a = tile_row_sum(colidx, s, e, Ct, NP / 4);
        if (p < npieces) reinterpret_cast<float4 *>(Ppc)[p * 8 + sub] = a;
    }
}

// long rows: P[row] = sum of the row's pieces, in order
__global__ void k_ppr_tile_fix(const int32_t *__restrict__ hub_rows, const int32_t *__restrict__ piece0, int32_t nh,
                               const float *__restrict__ Ppc, float *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t h = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; h < nh; h += nw) {
        float a = 0.0f;
        for (int32_t p = piece0[h]; p < piece0[h + 1]; ++p) a += Ppc[(int64_t)p * 32 + lane];
        P[(int64_t)hub_rows[h] * 32 + lane] = a;
    }
}

// Four rows per warp: 8 lanes per row, one float4 each (the tile's 32 columns = 128 bytes), and
// four in-edges in flight per row, so that every warp keeps 16 segment loads outstanding.
__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_gather(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx, int64_t R,
                                                                const float *__restrict__ C, int32_t NP, int32_t t,
                                                                float *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7, slot = lane >> 3;  // 4 rows per warp, 8 lanes per row
    const int64_t nw = (int64_t)gridDim.x * PT_WARPS;
    const float4 *Ct = reinterpret_cast<const float4 *>(C + 32 * t) + sub;
    const int64_t NP4 = NP / 4;
    for (int64_t r0 = ((int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5)) * 4; r0 < R; r0 += nw * 4) {
        const int64_t r = r0 + slot;
        int32_t s = 0, e = 0;
        if (r < R) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
        }
        const bool longrow = e - s > PT_PIECE;  // finished from its pieces
        const float4 a = tile_row_sum(colidx, s, longrow ? s : e, Ct, NP4);
        if (r < R && !longrow) reinterpret_cast<float4 *>(P)[r * 8 + sub] = a;
    }
}

__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_merge(const float *__restrict__ P,
                                                               const int32_t *__restrict__ id_map,
                                                               const int32_t *__restrict__ merge_off, int32_t B,
                                                               int32_t nranges, int32_t k, int32_t V, int32_t NP,
                                                               int32_t t, const int32_t *__restrict__ src_of_col,
                                                               const unsigned long long *__restrict__ Dcur,
                                                               unsigned long long *Dnext, unsigned long long *Dzero,
                                                               const float *__restrict__ inv_outdeg, float damping,
                                                               float *Cn, float *R_out, int32_t n) {
    extern __shared__ float pacc[];  // [k][32]
    __shared__ float dsh[PT_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j = blockIdx.x;
    const int32_t vbase = j * k;
    if (blockIdx.x == 0 && t == 0)
        for (int q = threadIdx.x; q < NP; q += PT_THREADS) Dzero[q] = 0ull;
    for (int q = threadIdx.x; q < k * 32; q += PT_THREADS) pacc[q] = 0.0f;
    __syncthreads();
    for (int32_t b = 0; b < B; ++b) {  // blocks in order: every vertex's sum has a fixed order
        const int32_t *o = merge_off + (int64_t)b * (nranges + 1) + j;
        const int32_t r0 = __ldg(o), r1 = __ldg(o + 1);
        for (int32_t r = r0 + warp; r < r1; r += PT_WARPS)
            pacc[(__ldg(id_map + r) - vbase) * 32 + lane] += __ldg(P + (int64_t)r * 32 + lane);
        __syncthreads();
    }
    const int32_t col = 32 * t + lane;
    const int32_t s = src_of_col[col];
    const float tele = (1.0f - damping) + damping * (float)((double)Dcur[col] / PPR_FX);
    float dl = 0.0f;
    for (int32_t q = warp; q < k; q += PT_WARPS) {
        const int32_t v = vbase + q;
        if (v >= V) break;
        const float r = damping * pacc[q * 32 + lane] + (s == v ? tele : 0.0f);
        const float inv = __ldg(inv_outdeg + v);
        Cn[(int64_t)v * NP + col] = r * inv;
        if (R_out && col < n) R_out[(int64_t)v * n + col] = r;
        if (inv == 0.0f) dl += r;
    }
    dsh[warp][lane] = dl;
    __syncthreads();
    if (warp == 0) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < PT_WARPS; ++w) tot += dsh[w][lane];
        if (tot != 0.0f) atomicAdd(Dnext + col, (unsigned long long)__double2ll_rn((double)tot * PPR_FX));
    }
}

struct Hubs {
    const int32_t *rows, *piece0;
    const int2 *pieces;
    int32_t nhubs, npieces;
    float *Ppc;
};

__global__ void k_row_bounds(const int32_t *rowptr, const int32_t *rows, int32_t n, int32_t *out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[2 * i] = rowptr[rows[i]];
        out[2 * i + 1] = rowptr[rows[i] + 1];
    }
}

// Pieces of the rows above `piece` edges: host-built from the hub list (few rows).
static int build_pieces(const int32_t *rowptr, const int32_t *hub_list, int32_t nh, int32_t NP, DevBuf *rows,
                        DevBuf *piece0, DevBuf *pieces, DevBuf *Ppc, Hubs *h, cudaStream_t s,
                        int32_t piece = PPR_PIECE) {
    h->nhubs = 0;
    h->npieces = 0;
    h->rows = nullptr;
    h->piece0 = nullptr;
    h->pieces = nullptr;
    h->Ppc = nullptr;
    if (nh <= 0) return TC_OK;
    int32_t *hl = new (std::nothrow) int32_t[nh];
    int32_t *rs = new (std::nothrow) int32_t[2 * (size_t)nh];
    if (!hl || !rs) {
        delete[] hl;
        delete[] rs;
        return fail(TC_ERR_OOM, "host allocation failed");
    }
    DevBuf bounds;
    int brc = bounds.alloc((size_t)nh * 8);
    if (brc != TC_OK) {
        delete[] hl;
        delete[] rs;
        return brc;
    }
    k_row_bounds<<<(nh + 255) / 256, 256, 0, s>>>(rowptr, hub_list, nh, bounds.as<int32_t>());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hl, hub_list, (size_t)nh * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rs, bounds.p, (size_t)nh * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete[] hl;
        delete[] rs;
        return fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    }
    int32_t *p0 = new (std::nothrow) int32_t[nh + 1];
    int64_t np = 0;
    for (int32_t i = 0; i < nh; ++i) np += (rs[2 * i + 1] - rs[2 * i] + piece - 1) / piece;
    int2 *pc = new (std::nothrow) int2[np > 0 ? np : 1];
    if (!p0 || !pc) {
        delete[] hl;
        delete[] rs;
        delete[] p0;
        delete[] pc;
        return fail(TC_ERR_OOM, "host allocation failed");
    }
    int64_t q = 0;
    for (int32_t i = 0; i < nh; ++i) {
        p0[i] = (int32_t)q;
        for (int32_t st = rs[2 * i]; st < rs[2 * i + 1]; st += piece) pc[q++] = make_int2(hl[i], st);
    }
    p0[nh] = (int32_t)q;
    int rc = rows->alloc((size_t)nh * 4);
    if (rc == TC_OK) rc = piece0->alloc((size_t)(nh + 1) * 4);
    if (rc == TC_OK) rc = pieces->alloc((size_t)(np > 0 ? np : 1) * 8);
    if (rc == TC_OK) rc = Ppc->alloc((size_t)(np > 0 ? np : 1) * NP * 4);
    if (rc == TC_OK) {
        e = cudaMemcpyAsync(rows->p, hl, (size_t)nh * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(piece0->p, p0, (size_t)(nh + 1) * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pieces->p, pc, (size_t)np * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    }
    delete[] hl;
    delete[] rs;
    delete[] p0;
    delete[] pc;
    if (rc != TC_OK) return rc;
    h->nhubs = nh;
    h->npieces = (int32_t)np;
    h->rows = rows->as<int32_t>();
    h->piece0 = piece0->as<int32_t>();
    h->pieces = pieces->as<int2>();
    h->Ppc = Ppc->as<float>();
    return TC_OK;
}

// The column-tiled TOCAB form (a pull partition in the graph's own numbering).
static int ppr_tiles_impl(const tc_graph *cg, const tc_part *part, const int32_t *sources, int32_t n,
                    const tc_pr_params *pp, float *R_out, tc_pr_stats *stats, cudaStream_t s) {
    tc_graph *g = const_cast<tc_graph *>(cg);
    const int32_t V = g->V;
    int NV4 = 1;
    while (128 * NV4 < n) NV4 *= 2;
    const int32_t NP = 128 * NV4;
    const size_t mat = (size_t)V * NP * 4;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    DevBuf Cbuf, srcbuf, Dbuf, Rdev;
    TC_TRY(Cbuf.alloc(2 * mat));
    TC_TRY(srcbuf.alloc((size_t)NP * 4));
    TC_TRY(Dbuf.alloc((size_t)3 * NP * 8));
    float *Cm[2] = {Cbuf.as<float>(), Cbuf.as<float>() + (size_t)V * NP};
    unsigned long long *D[3] = {Dbuf.as<unsigned long long>(), Dbuf.as<unsigned long long>() + NP,
                                Dbuf.as<unsigned long long>() + 2 * NP};
    int32_t *hsrc = new (std::nothrow) int32_t[NP];
    if (!hsrc) return fail(TC_ERR_OOM, "host allocation failed");
    for (int32_t j = 0; j < NP; ++j) hsrc[j] = j < n ? sources[j] : -1;
    cudaError_t e = cudaMemcpyAsync(srcbuf.p, hsrc, (size_t)NP * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] hsrc;
    if (e != cudaSuccess) return fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    float *Rd = R_out;
    if (pp->out_mem == TC_MEM_HOST) {
        TC_TRY(Rdev.alloc((size_t)V * n * 4));
        Rd = Rdev.as<float>();
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (pp->profile) {
        TC_CUDA(cudaEventCreate(&ev[0]));
        TC_CUDA(cudaEventCreate(&ev[1]));
        TC_CUDA(cudaEventRecord(ev[0], s));
    }
    TC_CUDA(cudaMemsetAsync(Cm[0], 0, mat, s));
    if (pp->iters == 0) TC_CUDA(cudaMemsetAsync(Rd, 0, (size_t)V * n * 4, s));
    k_ppr_init<<<(NP + 255) / 256, 256, 0, s>>>(Cm[0], NP, srcbuf.as<int32_t>(), g->inv_outdeg.as<float>(), D[0],
                                                pp->iters == 0 ? Rd : nullptr, n);
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaMemsetAsync(D[1], 0, (size_t)NP * 8, s));
    int launches = 1;
    const int32_t ntiles = NP / 32;
    DevBuf Pbuf;
    size_t tm_smem = 0;
    int tg_grid = 1;
    Hubs th;
    DevBuf th_list, th_rows, th_p0, th_pcs, th_ppc;
    int32_t tnh = 0;
    if (part) {
        TC_TRY(collect_hubs(part->rowptr.as<int32_t>(), part->R, PT_PIECE, &th_list, &tnh, s));
        // piece partials are 32 floats: NP argument 32
        TC_TRY(build_pieces(part->rowptr.as<int32_t>(), th_list.as<int32_t>(), tnh, 32, &th_rows, &th_p0, &th_pcs,
                            &th_ppc, &th, s, PT_PIECE));
        TC_TRY(Pbuf.alloc((size_t)(part->R > 0 ? part->R : 1) * 32 * 4));
        tm_smem = (size_t)part->k * 32 * 4;
        TC_CUDA(cudaFuncSetAttribute(k_ppr_tile_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tm_smem));
        int ps = 1;
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_ppr_tile_gather, PT_THREADS, 0));
        tg_grid = caps.sms * (ps > 0 ? ps : 1);
    }
    for (int it = 0; it < pp->iters; ++it) {
        const bool last = it == pp->iters - 1;
        const float *Cc = Cm[it & 1];
        float *Cn = Cm[(it + 1) & 1];
        unsigned long long *Dc = D[it % 3], *Dn = D[(it + 1) % 3], *Dz = D[(it + 2) % 3];
        for (int32_t t = 0; t < ntiles; ++t) {
            if (th.npieces > 0) {
                k_ppr_tile_piece<<<tg_grid, PT_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                                th.pieces, th.npieces, Cc, NP, t, th.Ppc);
                ++launches;
            }
            k_ppr_tile_gather<<<tg_grid, PT_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                             part->R, Cc, NP, t, Pbuf.as<float>());
            if (th.nhubs > 0) {
                k_ppr_tile_fix<<<(th.nhubs * 32 + 255) / 256, 256, 0, s>>>(th.rows, th.piece0, th.nhubs, th.Ppc,
                                                                          Pbuf.as<float>());
                ++launches;
            }
            k_ppr_tile_merge<<<part->nranges, PT_THREADS, tm_smem, s>>>(
                Pbuf.as<float>(), part->id_map.as<int32_t>(), part->merge_off.as<int32_t>(), part->B, part->nranges,
                part->k, g->V, NP, t, srcbuf.as<int32_t>(), Dc, Dn, Dz, g->inv_outdeg.as<float>(), pp->damping,
                Cn, last ? Rd : nullptr, n);
            TC_LAUNCH_CHECK();
            launches += 2;
        }
    }
    float ms = 0;
    if (pp->profile) {
        TC_CUDA(cudaEventRecord(ev[1], s));
        TC_CUDA(cudaEventSynchronize(ev[1]));
        TC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (pp->out_mem == TC_MEM_HOST)
        TC_CUDA(cudaMemcpyAsync(R_out, Rd, (size_t)V * n * 4, cudaMemcpyDeviceToHost, s));
    // the scratch buffers are freed at return: finish their users first
    TC_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iters = pp->iters;
        stats->launches = launches;
        stats->ms_total = ms;
        stats->ms_gather = ms;
    }
    return TC_OK;
}

// ---------------------------------------------------------------------------------------------
// the persistent batch
// ---------------------------------------------------------------------------------------------
// The persistent kernel for NP padded columns and tile width tw (0: whole rows; 128, 64 or 32).
static const void *persist_kernel(int32_t NP, int32_t tw) {
    if (tw == 128) return (const void *)k_ppr_tiled<1>;
    if (tw == 64) return (const void *)k_ppr_tiled<2>;
    if (tw == 32) return (const void *)k_ppr_tiled<4>;
    const int NV4 = NP / 128;
    return NV4 == 1 ? (const void *)k_ppr_persist<1>
           : NV4 == 2 ? (const void *)k_ppr_persist<2>
           : NV4 == 4 ? (const void *)k_ppr_persist<4>
                      : (const void *)k_ppr_persist<8>;
}

// Dynamic shared memory of the whole-row kernel: the warps' fixed-point dangling sums.
static size_t persist_smem(int32_t NP, int32_t tw) { return tw ? 0 : (size_t)PPR_WARPS * NP * 8; }

// CTAs of the persistent kernel resident per SM.
static int persist_occupancy(int32_t NP, int32_t tw, int *per_sm) {
    const void *k = persist_kernel(NP, tw);
    const size_t smem = persist_smem(NP, tw);
    TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, PPR_THREADS, smem));
    return TC_OK;
}

// The numbering by out-degree of the graph, its buffers for NP padded columns, and the pieces of
// its long rows (rebuilt when NP changes).
static int ppr_prepare(tc_graph *g, int32_t NP, cudaStream_t s) {
    if (!g->ord_built) {
        TC_TRY(order_by_outdegree(g, s, &g->ord_perm, &g->ord_inv, &g->ord_inv_outdeg, &g->ord_rowptr, &g->ord_colidx,
                                  nullptr, &g->ord_ni));
        g->ord_built = true;
    }
    if (!g->ppr_light_built) {  // the light rows and their runs (independent of the column count)
        const int32_t V = g->V;
        DeviceCaps caps;
        TC_TRY(device_caps(&caps));
        DevBuf deg;
        TC_TRY(deg.alloc(((size_t)V + 1) * 4));
        TC_TRY(g->ppr_islong.alloc((size_t)V + 16));
        TC_TRY(g->ppr_rowptr_l.alloc(((size_t)V + 1) * 4));
        k_ppr_light_deg<<<caps.sms * 8, 256, 0, s>>>(g->ord_rowptr.as<int32_t>(), V, deg.as<int32_t>(),
                                                     g->ppr_islong.as<uint8_t>());
        TC_LAUNCH_CHECK();
        TC_TRY(scan_i32(deg.as<int32_t>(), (int64_t)V + 1, g->ppr_rowptr_l.as<int32_t>(), s));
        int32_t El = 0;
        TC_CUDA(cudaMemcpyAsync(&El, g->ppr_rowptr_l.as<int32_t>() + V, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        TC_TRY(g->ppr_colidx_l.alloc((size_t)(El > 0 ? El : 1) * 4 + 64));
        k_ppr_light_copy<<<caps.sms * 16, 256, 0, s>>>(g->ord_rowptr.as<int32_t>(), g->ord_colidx.as<int32_t>(), V,
                                                       g->ppr_rowptr_l.as<int32_t>(), g->ppr_colidx_l.as<int32_t>());
        TC_LAUNCH_CHECK();
        const int64_t total = (int64_t)El + (int64_t)PPR_ROW_COST * V;
        const int64_t nch = (total + PPR_SUB_COST - 1) / PPR_SUB_COST;
        g->ppr_nchunks = (int32_t)(nch > 0 ? nch : 1);
        TC_TRY(g->ppr_chunks.alloc(((size_t)g->ppr_nchunks + 1) * 4));
        k_ppr_chunks<<<(g->ppr_nchunks + 256) / 256, 256, 0, s>>>(g->ppr_rowptr_l.as<int32_t>(), V, PPR_SUB_COST,
                                                                  g->ppr_nchunks, g->ppr_chunks.as<int32_t>());
        TC_LAUNCH_CHECK();
        TC_CUDA(cudaStreamSynchronize(s));  // deg is freed at return
        g->ppr_light_built = true;
    }
    if (g->ppr_np == NP) return TC_OK;
    if (g->ppr_exec) {
        cudaGraphExecDestroy(g->ppr_exec);
        g->ppr_exec = nullptr;
    }
    g->ppr_np = 0;
    const int32_t V = g->V;
    TC_TRY(g->ppr_C.alloc((size_t)V * 2 * NP * 4 + 256));
    TC_TRY(g->ppr_D.alloc((size_t)3 * NP * 8));
    TC_TRY(g->ppr_src_old.alloc((size_t)NP * 4));
    TC_TRY(g->ppr_src.alloc((size_t)NP * 4));
    TC_TRY(g->ppr_isrc.alloc((size_t)V + 16));
    TC_TRY(g->ppr_sync.alloc(64));
    DevBuf hub_list;
    int32_t nh = 0;
    TC_TRY(collect_hubs(g->ord_rowptr.as<int32_t>(), V, PPR_PIECE, &hub_list, &nh, s));
    Hubs h;
    TC_TRY(build_pieces(g->ord_rowptr.as<int32_t>(), hub_list.as<int32_t>(), nh, NP, &g->ppr_hub_rows, &g->ppr_hub_p0,
                        &g->ppr_pieces, &g->ppr_Ppc, &h, s));
    if (h.nhubs == 0) {  // keep the arguments valid
        TC_TRY(g->ppr_hub_p0.alloc(16));
        TC_TRY(g->ppr_hub_rows.alloc(16));
        TC_TRY(g->ppr_pieces.alloc(16));
        TC_TRY(g->ppr_Ppc.alloc(16));
    }
    TC_TRY(g->ppr_hubcnt.alloc((size_t)(h.nhubs > 0 ? h.nhubs : 1) * 4));
    g->ppr_nhubs = h.nhubs;
    g->ppr_npieces = h.npieces;
    g->ppr_np = NP;
    return TC_OK;
}

// Largest hot block: as many rows of `width` columns as the L2 holds.
static int ppr_max_hot(const tc_graph *g, int32_t width, int32_t *hot) {
    int dev = 0, l2 = 0;
    TC_CUDA(cudaGetDevice(&dev));
    TC_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    int64_t h = (int64_t)l2 / ((int64_t)width * 4);
    if (h > g->V) h = g->V;
    *hot = (int32_t)(h > 0 ? h : 0);
    return TC_OK;
}

// The whole call as one stream sequence: columns, matrix 0, then the persistent kernel (whose
// accesses to the rows of the first `hot` sources are evict-last).
static int ppr_launch(tc_graph *g, int32_t n, const tc_pr_params *pp, float *R_out, int32_t hot, int32_t tw, int grid,
                      cudaStream_t s) {
    const int32_t NP = g->ppr_np, V = g->V;
    unsigned long long *D = g->ppr_D.as<unsigned long long>();
    TC_CUDA(cudaMemsetAsync(g->ppr_isrc.p, 0, (size_t)V, s));
    TC_CUDA(cudaMemsetAsync(D, 0, (size_t)3 * NP * 8, s));
    TC_CUDA(cudaMemsetAsync(g->ppr_sync.p, 0, 32, s));  // barrier, error flag, queue heads
    TC_CUDA(cudaMemsetAsync(g->ppr_hubcnt.p, 0, (size_t)(g->ppr_nhubs > 0 ? g->ppr_nhubs : 1) * 4, s));
    k_ppr_columns<<<(NP + 255) / 256, 256, 0, s>>>(g->ppr_src_old.as<int32_t>(), n, NP, g->ord_inv.as<int32_t>(),
                                                   g->ord_inv_outdeg.as<float>(), g->ppr_src.as<int32_t>(),
                                                   g->ppr_isrc.as<uint8_t>(), D);
    TC_LAUNCH_CHECK();
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    k_ppr_clear0<<<caps.sms * 8, 256, 0, s>>>(g->ppr_C.as<float4>(), V, NP);
    TC_LAUNCH_CHECK();
    k_ppr_seed<<<(NP + 255) / 256, 256, 0, s>>>(g->ppr_C.as<float>(), NP, g->ppr_src.as<int32_t>(),
                                                g->ord_inv_outdeg.as<float>());
    TC_LAUNCH_CHECK();
    PprArgs a;
    a.rowptr = g->ord_rowptr.as<int32_t>();
    a.colidx = g->ord_colidx.as<int32_t>();
    a.rowptr_l = g->ppr_rowptr_l.as<int32_t>();
    a.colidx_l = g->ppr_colidx_l.as<int32_t>();
    a.chunk_row = g->ppr_chunks.as<int32_t>();
    a.nsub = g->ppr_nchunks;
    a.V = V;
    a.np = NP;
    a.n = n;
    a.iters = pp->iters;
    a.CC = g->ppr_C.as<float>();
    a.srcc = g->ppr_src.as<int32_t>();
    a.D = D;
    a.inv_outdeg = g->ord_inv_outdeg.as<float>();
    a.damping = pp->damping;
    a.R_out = R_out;
    a.perm = g->ord_perm.as<int32_t>();
    a.is_src = g->ppr_isrc.as<uint8_t>();
    a.is_long = g->ppr_islong.as<uint8_t>();
    a.hub_rows = g->ppr_hub_rows.as<int32_t>();
    a.hub_piece0 = g->ppr_hub_p0.as<int32_t>();
    a.pieces = g->ppr_pieces.as<int2>();
    a.nhubs = g->ppr_nhubs;
    a.npieces = g->ppr_npieces;
    a.Ppc = g->ppr_Ppc.as<float>();
    a.hub_count = g->ppr_hubcnt.as<unsigned>();
    a.hot = hot;
    a.sync = g->ppr_sync.as<unsigned>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(PPR_THREADS);
    cfg.dynamicSmemBytes = persist_smem(NP, tw);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[1] = {&a};
    TC_CUDA(cudaLaunchKernelExC(&cfg, persist_kernel(NP, tw), args));
    return TC_OK;
}

// The persistent batch: hot < 0 and tw < 0 take the tuned (or default) choices.
static int ppr_persist_impl(tc_graph *g, const int32_t *sources, int32_t n, const tc_pr_params *pp, float *R_out,
                            tc_pr_stats *stats, int32_t hot, int32_t tw, bool use_graph, cudaStream_t s) {
    const int32_t V = g->V;
    int NV4 = 1;
    while (128 * NV4 < n) NV4 *= 2;
    const int32_t NP = 128 * NV4;
    float *Rd = R_out;
    DevBuf Rdev;
    if (pp->out_mem == TC_MEM_HOST) {
        TC_TRY(Rdev.alloc((size_t)V * n * 4));
        Rd = Rdev.as<float>();
    }
    if (pp->iters == 0) {  // R = e_s (caller's IDs)
        TC_CUDA(cudaMemsetAsync(Rd, 0, (size_t)V * n * 4, s));
        DevBuf sb;
        TC_TRY(sb.alloc((size_t)n * 4));
        TC_CUDA(cudaMemcpyAsync(sb.p, sources, (size_t)n * 4, cudaMemcpyHostToDevice, s));
        k_ppr_unit<<<(n + 255) / 256, 256, 0, s>>>(sb.as<int32_t>(), n, Rd);
        TC_LAUNCH_CHECK();
        TC_CUDA(cudaStreamSynchronize(s));  // sb is freed at the end of this block
    } else {
        TC_TRY(ppr_prepare(g, NP, s));
        if (tw < 0) tw = g->ppr_tile >= 0 ? g->ppr_tile : PPR_DEFAULT_TILE;
        if (tw != 0 && tw != 32 && tw != 64 && tw != 128) return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: bad tile width");
        int32_t hmax = 0;
        TC_TRY(ppr_max_hot(g, tw ? tw : NP, &hmax));
        if (hot < 0) hot = g->ppr_hot >= 0 ? g->ppr_hot : hmax / 2;
        if (hot > hmax) hot = hmax;
        DeviceCaps caps;
        TC_TRY(device_caps(&caps));
        int per_sm = 0;
        TC_TRY(persist_occupancy(NP, tw, &per_sm));
        if (per_sm < 1) return fail(TC_ERR_CUDA, "tc_ppr_batch: the persistent kernel cannot be resident");
        const int grid = caps.sms * per_sm;
        TC_CUDA(cudaMemcpyAsync(g->ppr_src_old.p, sources, (size_t)n * 4, cudaMemcpyHostToDevice, s));
        cudaEvent_t ev[2] = {nullptr, nullptr};
        if (pp->profile) {
            TC_CUDA(cudaEventCreate(&ev[0]));
            TC_CUDA(cudaEventCreate(&ev[1]));
            TC_CUDA(cudaEventRecord(ev[0], s));
        }
        if (!use_graph) {
            TC_TRY(ppr_launch(g, n, pp, Rd, hot, tw, grid, s));
        } else {
            const bool same = g->ppr_exec && g->ppr_key_out == Rd && g->ppr_key_n == n && g->ppr_key_iters == pp->iters &&
                              g->ppr_key_damping == pp->damping && g->ppr_key_hot == hot && g->ppr_key_grid == grid &&
                              g->ppr_key_tile == tw;
            if (!same) {
                if (g->ppr_exec) {
                    cudaGraphExecDestroy(g->ppr_exec);
                    g->ppr_exec = nullptr;
                }
                cudaStream_t cs;
                TC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                cudaGraph_t graph = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                int st = TC_OK;
                if (e == cudaSuccess) {
                    st = ppr_launch(g, n, pp, Rd, hot, tw, grid, cs);
                    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                    if (e == cudaSuccess) e = e2;
                }
                if (e == cudaSuccess && st == TC_OK) e = cudaGraphInstantiate(&g->ppr_exec, graph, 0);
                if (graph) cudaGraphDestroy(graph);
                cudaStreamDestroy(cs);
                if (st != TC_OK) return st;
                if (e != cudaSuccess) {
                    g->ppr_exec = nullptr;
                    return fail(TC_ERR_CUDA, "tc_ppr_batch: capturing the persistent launch failed: %s",
                                cudaGetErrorString(e));
                }
                g->ppr_key_out = Rd;
                g->ppr_key_n = n;
                g->ppr_key_iters = pp->iters;
                g->ppr_key_damping = pp->damping;
                g->ppr_key_hot = hot;
                g->ppr_key_grid = grid;
                g->ppr_key_tile = tw;
            }
            TC_CUDA(cudaGraphLaunch(g->ppr_exec, s));
        }
        float ms = 0;
        if (pp->profile) {
            TC_CUDA(cudaEventRecord(ev[1], s));
            TC_CUDA(cudaEventSynchronize(ev[1]));
            TC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
            cudaEventDestroy(ev[0]);
            cudaEventDestroy(ev[1]);
        }
        int err = 0;
        TC_CUDA(cudaMemcpyAsync(&err, g->ppr_sync.as<unsigned>() + 2, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        if (err) return fail(TC_ERR_TIMEOUT, "tc_ppr_batch: a grid barrier gave up");
        if (stats) {
            memset(stats, 0, sizeof(*stats));
            stats->iters = pp->iters;
            stats->launches = 1;
            stats->ms_total = ms;
            stats->ms_gather = ms;
        }
    }
    if (pp->out_mem == TC_MEM_HOST) TC_CUDA(cudaMemcpyAsync(R_out, Rd, (size_t)V * n * 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (stats && pp->iters == 0) memset(stats, 0, sizeof(*stats));
    return TC_OK;
}

static int ppr_impl(const tc_graph *cg, const tc_part *part, const int32_t *sources, int32_t n,
                    const tc_pr_params *pp, float *R_out, tc_pr_stats *stats, cudaStream_t s) {
    if (part) return ppr_tiles_impl(cg, part, sources, n, pp, R_out, stats, s);
    return ppr_persist_impl(const_cast<tc_graph *>(cg), sources, n, pp, R_out, stats, -1, -1, true, s);
}

}  // namespace tc

extern "C" int tc_ppr_autotune(tc_graph *g, const int32_t *sources, int32_t n, const tc_pr_params *params,
                               int32_t *best_hot, int32_t *best_tile, float *times, void *stream) {
    using namespace tc;
    if (!g || !sources || !params || n < 1 || n > 1024) return fail(TC_ERR_INVALID_ARG, "tc_ppr_autotune: bad argument");
    if (!(params->damping >= 0.0f && params->damping <= 1.0f))
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_autotune: damping outside [0,1]");
    for (int32_t j = 0; j < n; ++j)
        if (sources[j] < 0 || sources[j] >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_ppr_autotune: source outside [0, V)");
    cudaStream_t s = (cudaStream_t)stream;
    int NV4 = 1;
    while (128 * NV4 < n) NV4 *= 2;
    const int32_t NP = 128 * NV4;
    TC_TRY(ppr_prepare(g, NP, s));
    DevBuf R;
    TC_TRY(R.alloc((size_t)g->V * n * 4));
    tc_pr_params pp = *params;
    pp.out_mem = TC_MEM_DEVICE;
    pp.profile = 1;
    if (pp.iters <= 0 || pp.iters > 3) pp.iters = 3;  // a few iterations tell the variants apart
    // tile widths (0: whole rows) x evict-last rows (0, 1/4, 1/2 and all of the rows the L2 holds)
    const int32_t tws[4] = {0, 128, 64, 32};
    const int32_t num[4] = {0, 1, 2, 4};
    float best = 0.0f;
    int32_t bh = 0, bt = 0;
    for (int ti = 0; ti < 4; ++ti) {
        int32_t hmax = 0;
        TC_TRY(ppr_max_hot(g, tws[ti] ? tws[ti] : NP, &hmax));
        for (int hi = 0; hi < 4; ++hi) {
            const int32_t hot = (int32_t)((int64_t)hmax * num[hi] / 4);
            tc_pr_stats st;
            TC_TRY(ppr_persist_impl(g, sources, n, &pp, R.as<float>(), nullptr, hot, tws[ti], false, s));  // warm
            TC_TRY(ppr_persist_impl(g, sources, n, &pp, R.as<float>(), &st, hot, tws[ti], false, s));
            if (times) times[ti * 4 + hi] = st.ms_total;
            if ((ti == 0 && hi == 0) || st.ms_total < best) {
                best = st.ms_total;
                bh = hot;
                bt = tws[ti];
            }
        }
    }
    g->ppr_hot = bh;
    g->ppr_tile = bt;
    if (best_hot) *best_hot = bh;
    if (best_tile) *best_tile = bt;
    return TC_OK;
}

extern "C" int tc_ppr_set_tuning(tc_graph *g, int32_t hot, int32_t tile) {
    using namespace tc;
    if (!g || hot < -1 || (tile != -1 && tile != 0 && tile != 32 && tile != 64 && tile != 128))
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_set_tuning: bad argument");
    g->ppr_hot = hot;
    g->ppr_tile = tile;
    return TC_OK;
}

extern "C" int tc_ppr_batch(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t n,
                            const tc_pr_params *params, float *R_out, tc_pr_stats *stats, void *stream) {
    using namespace tc;
    if (!g || !sources || !params || !R_out) return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: null argument");
    if (part && (part->g != g || part->dir != TC_PULL))
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: partition must be a TC_PULL partition of this graph");
    if (part && part->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if (part && (size_t)part->k * 32 * 4 > 200 * 1024)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: the partition's merge_range must be <= 1600 (<= 256 advised)");
    if (n < 1 || n > 1024) return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: n must be in [1, 1024]");
    if (!(params->damping >= 0.0f && params->damping <= 1.0f) || params->iters < 0)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: damping outside [0,1] or iters < 0");
    if (params->out_mem != TC_MEM_HOST && params->out_mem != TC_MEM_DEVICE)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: bad out_mem");
    for (int32_t j = 0; j < n; ++j)
        if (sources[j] < 0 || sources[j] >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: source %d outside [0, V)", j);
    if ((int64_t)g->V * ((n + 127) / 128 * 128) * 8 > ((int64_t)1 << 40))
        return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: V x n too large");
    return ppr_impl(g, part, sources, n, params, R_out, stats, (cudaStream_t)stream);
}
