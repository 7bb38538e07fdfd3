// PageRank iteration kernels and drivers.
//   pull, unblocked : Alg. 1 with the update fused into the gather epilogue.
//   pull, TOCAB     : Alg. 4 per block into partial sums over local IDs, then the merge of
//                     Fig. 5 (one CTA per vertex range) fused with the update.
//   push            : Alg. 2 / Alg. 5 atomic scatter, then a separate update kernel.
// Load balancing (Sec. 3.2): a warp takes 32 consecutive rows; rows with fewer than 32
// edges are summed serially by their lane, rows up to the hub degree by the whole warp,
// and hub rows by a whole CTA each (thread / warp / CTA per row, no atomics in pull).
#include "tc_common_dev.cuh"

namespace tc {

constexpr int PR_THREADS = 256;
constexpr int PR_WARPS = PR_THREADS / 32;

struct UpdateArgs {
    float base;             // (1-d)/V
    float damping;          // d
    int drop;               // 1: dangling mass is not redistributed
    int32_t V;
    const double *D_cur;    // dangling mass of the ranks the current contributions came from
    double *D_next;         // dangling mass of the ranks written now
    double *dpart;          // per-CTA partial dangling sums
    unsigned *counter;      // arrival counter for the last-CTA reduction
    const float *inv_outdeg;
    float *rank_out;        // may be null (only the last iteration writes ranks)
    float *contrib_next;    // contributions for the next iteration
    double *fx_scale;       // fixed-point scale of the merge (written by the init kernel)
    const int32_t *perm;    // renumbered partitions: original ID of vertex v (null: identity)
    int32_t nz;             // renumbered: vertices [nz, V) have no out-edges (else nz = V)
    int32_t ni;             // renumbered: vertices [ni, V) have no edge at all (else ni = V)
    int *err;               // sticky error flag of bounded device waits
    unsigned *queue;        // work queue of the persistent merge (zero between launches)
    // direct pieces of the partition (null when it has none): per merge range j, pieces
    // [dir_off[j], dir_off[j+1]) add cur[dir_u[i]] to vertex rstart[j] + dir_id16[i]
    const int32_t *dir_off;
    const int32_t *dir_u;
    const uint16_t *dir_id16;
    const float *cur;       // the contributions the gather read
};

__device__ __forceinline__ float spread_of(const UpdateArgs &u) {
    return u.drop ? 0.0f : (float)(*u.D_cur / (double)u.V);
}

// rank[v] = (1-d)/V + d (sum + D/V); contribution = rank / out_degree; returns the dangling share.
// Ranks leave under the caller's vertex IDs.  Renumbered vertices from nz on have no out-edges:
// their contribution is never read, so neither the reciprocal is loaded nor the value stored.
__device__ __forceinline__ float apply_update(const UpdateArgs &u, int32_t v, float sum, float spread) {
    const float r = u.base + u.damping * (sum + spread);
    if (u.rank_out) u.rank_out[u.perm ? __ldg(u.perm + v) : v] = r;
    if (v >= u.nz) return r;
    const float inv = __ldg(u.inv_outdeg + v);
    u.contrib_next[v] = r * inv;
    return inv == 0.0f ? r : 0.0f;
}

// The same update with the out-degree reciprocal of v already at hand (inv; ignored from nz on).
__device__ __forceinline__ float apply_update_inv(const UpdateArgs &u, int32_t v, float sum, float spread, float inv) {
    const float r = u.base + u.damping * (sum + spread);
    if (u.rank_out) u.rank_out[u.perm ? __ldg(u.perm + v) : v] = r;
    if (v >= u.nz) return r;
    u.contrib_next[v] = r * inv;
    return inv == 0.0f ? r : 0.0f;
}

// ---------------------------------------------------------------------------------------------
// Pull gather over a CSR whose rows are destinations (G^T, or the TOCAB row space).
// FUSED = true: rows are vertices, apply the update; FUSED = false: write partial[row].
// ---------------------------------------------------------------------------------------------
// Load-balancing knobs (Sec. 3.2): rows with fewer than warp_min edges are summed by one lane,
// rows up to hub_degree by the whole warp, larger rows by a whole CTA.  With a per-block table
// (lb_tab[b], blocks found through blk_rows) every TOCAB subgraph has its own warp_min.
struct LbArgs {
    int32_t warp_min;
    const int32_t *lb_tab;   // null: warp_min everywhere
    const int64_t *blk_rows; // [B+1]
    int32_t B;
};

__device__ __forceinline__ int32_t lb_warp_min(const LbArgs &lb, int64_t row) {
    if (!lb.lb_tab) return lb.warp_min;
    int32_t lo = 0, hi = lb.B;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (__ldg(lb.blk_rows + mid) <= row) lo = mid; else hi = mid;
    }
    return __ldg(lb.lb_tab + lo);
}

template <bool FUSED>
__global__ void __launch_bounds__(PR_THREADS) k_pull_gather(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx, int64_t nrows,
                                                            const int32_t *__restrict__ hubs, int32_t num_hubs,
                                                            int32_t hub_degree, int hub_ctas,
                                                            const float *__restrict__ contrib,
                                                            float *__restrict__ partial, UpdateArgs u, LbArgs lb) {
    __shared__ float fred[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float dsum = 0.0f;
    float spread = 0.0f;
    if (FUSED) spread = spread_of(u);
    if ((int)blockIdx.x < hub_ctas) {
        for (int32_t h = blockIdx.x; h < num_hubs; h += hub_ctas) {
            const int32_t row = hubs[h];
            const int32_t s = rowptr[row], e = rowptr[row + 1];
            float acc = 0.0f;
            for (int32_t i = s + threadIdx.x; i < e; i += PR_THREADS) acc += __ldg(contrib + __ldg(colidx + i));
            acc = block_sum<float>(acc, fred);
            if (threadIdx.x == 0) {
                if (FUSED) dsum += apply_update(u, row, acc, spread);
                else partial[row] = acc;
            }
        }
    } else {
        const int64_t ngroups = (nrows + 31) >> 5;
        const int64_t nwarps = (int64_t)(gridDim.x - hub_ctas) * PR_WARPS;
        for (int64_t grp = (int64_t)(blockIdx.x - hub_ctas) * PR_WARPS + warp; grp < ngroups; grp += nwarps) {
            const int64_t row = grp * 32 + lane;
            const bool valid = row < nrows;
            int32_t s = 0, e = 0;
            if (valid) {
                s = __ldg(rowptr + row);
                e = __ldg(rowptr + row + 1);
            }
            const int32_t deg = e - s;
            const int32_t wmin = lb_warp_min(lb, grp * 32);
            float sum = 0.0f;
            if (deg < wmin && deg <= hub_degree) {  // thread per row (hubs go to their CTA)
                for (int32_t i = s; i < e; ++i) sum += __ldg(contrib + __ldg(colidx + i));
            }
            unsigned wm = __ballot_sync(0xffffffffu, valid && deg >= wmin && deg <= hub_degree);
            while (wm) {  // warp per row
                const int l = __ffs(wm) - 1;
                wm &= wm - 1;
                const int32_t ws = __shfl_sync(0xffffffffu, s, l), we = __shfl_sync(0xffffffffu, e, l);
                float acc = 0.0f;
                for (int32_t i = ws + lane; i < we; i += 32) acc += __ldg(contrib + __ldg(colidx + i));
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
                if (lane == l) sum = acc;
            }
            if (valid && deg <= hub_degree) {
                if (FUSED) dsum += apply_update(u, (int32_t)row, sum, spread);
                else partial[row] = sum;
            }
        }
    }
    if (FUSED) {
        const float bs = block_sum<float>(dsum, fred);
        grid_sum_last_cta((double)bs, u.dpart, u.counter, u.D_next);
    }
}

// ---------------------------------------------------------------------------------------------
// TOCAB merge (Fig. 5): CTA j owns vertices [j*k, (j+1)*k).  For every block it reads the slice
// of local rows whose global IDs fall in the range (bounds from the range-major table).  The
// slices are cut into chunks of at most 32 rows; warp w takes chunks w, w+16, ... of the
// flattened chunk list, several at a time, and adds them into its own shared-memory
// accumulator (the rows of one chunk have distinct IDs, so no atomics are needed).  The 16
// accumulators are then added in warp order: the summation order is fixed, so the merge is
// deterministic.  The rank update of Alg. 1, the next contributions and the dangling
// mass are fused in.
// ---------------------------------------------------------------------------------------------
constexpr int MG_THREADS = 512;
constexpr int MG_WARPS = MG_THREADS / 32;
constexpr int MG_UNROLL = 16;
constexpr int MG_CMAP_EXTRA = 1024;  // chunk-to-block map entries beyond one per block

size_t merge_smem_bytes(int32_t k, int32_t B) {
    return (size_t)MG_WARPS * k * 4 + ((size_t)3 * B + 2) * 4 + ((size_t)B + MG_CMAP_EXTRA) * 2;
}

// id16 != null: local id inside the range is id16[r] (k a power of two <= 65536);
// otherwise id_map[r] - j*k.
__global__ void __launch_bounds__(MG_THREADS) k_pull_merge_ordered(const float *__restrict__ partial,
                                                           const int32_t *__restrict__ id_map,
                                                           const uint16_t *__restrict__ id16,
                                                           const int32_t *__restrict__ offT, int32_t B, int32_t k,
                                                           const int32_t *__restrict__ rstart, UpdateArgs u) {
    extern __shared__ __align__(16) unsigned char msm[];
    float *acc = reinterpret_cast<float *>(msm);                        // [MG_WARPS][k]
    int32_t *lo = reinterpret_cast<int32_t *>(acc + (size_t)MG_WARPS * k);  // [B]
    int32_t *len = lo + B;                                              // [B]
    int32_t *cpre = len + B;                                            // [B + 1] chunk prefix
    uint16_t *cmap = reinterpret_cast<uint16_t *>(cpre + B + 1);        // [B + MG_CMAP_EXTRA]
    const int32_t cmap_cap = B + MG_CMAP_EXTRA;
    __shared__ int32_t wsum[MG_WARPS];
    __shared__ float fred[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t j = blockIdx.x;
    // range j: [j k, (j+1) k), or [rstart[j], rstart[j+1]) (at most k wide) when given
    const int32_t vbase = rstart ? rstart[j] : j * k;
    const int32_t width = rstart ? rstart[j + 1] - vbase : k;
    for (int t = tid; t < MG_WARPS * k; t += MG_THREADS) acc[t] = 0.0f;
    // slice bounds and chunk counts of every block, then an exclusive scan of the counts
    const int per = (B + MG_THREADS - 1) / MG_THREADS;
    int32_t run = 0;
    for (int q = 0; q < per; ++q) {
        const int32_t b = tid * per + q;
        if (b < B) {
            const int32_t l0 = __ldg(offT + (int64_t)j * B + b), l1 = __ldg(offT + (int64_t)(j + 1) * B + b);
            lo[b] = l0;
            len[b] = l1 - l0;
            run += (l1 - l0 + 31) >> 5;
        }
    }
    int incl = run;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int w = lane < MG_WARPS ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < MG_WARPS) wsum[lane] = wi - w;
    }
    __syncthreads();
    int32_t base = wsum[warp] + incl - run;
    for (int q = 0; q < per; ++q) {
        const int32_t b = tid * per + q;
        if (b < B) {
            cpre[b] = base;
            base += (len[b] + 31) >> 5;
        }
    }
    if (tid == MG_THREADS - 1) cpre[B] = base;
    __syncthreads();
    // chunk -> block map (B <= 65535 here); chunks past its capacity are found by walking
    for (int q = 0; q < per; ++q) {
        const int32_t b = tid * per + q;
        if (b < B)
            for (int32_t c = cpre[b]; c < cpre[b + 1] && c < cmap_cap; ++c) cmap[c] = (uint16_t)b;
    }
    __syncthreads();
    const int32_t nchunks = cpre[B];
    float *mine = acc + (size_t)warp * k;
    for (int32_t c0 = warp; c0 < nchunks; c0 += MG_WARPS * MG_UNROLL) {
        int32_t idq[MG_UNROLL];
        float vq[MG_UNROLL];
#pragma unroll
        for (int q = 0; q < MG_UNROLL; ++q) {
            const int32_t c = c0 + q * MG_WARPS;
            idq[q] = -1;
            vq[q] = 0.0f;
            if (c < nchunks) {
                int32_t bp;
                if (c < cmap_cap) {
                    bp = cmap[c];
                } else {
                    bp = cmap[cmap_cap - 1];
                    while (cpre[bp + 1] <= c) ++bp;
                }
                const int32_t i = ((c - cpre[bp]) << 5) + lane;
                if (i < len[bp]) {
                    const int32_t r = lo[bp] + i;
                    idq[q] = id16 ? (int32_t)__ldg(id16 + r) : __ldg(id_map + r) - vbase;
                    vq[q] = __ldg(partial + r);
                }
            }
        }
        // one chunk at a time: rows of a chunk have distinct IDs; chunks may share IDs
#pragma unroll
        for (int q = 0; q < MG_UNROLL; ++q) {
            if (idq[q] >= 0) mine[idq[q]] += vq[q];
            __syncwarp();
        }
    }
    if (u.dir_off) {  // direct pieces, 32 per warp step; their targets ascend, so equal targets
                      // are adjacent lanes: a segmented sum, then the segment's last lane adds
        const int32_t d0 = __ldg(u.dir_off + j), d1 = __ldg(u.dir_off + j + 1);
        for (int32_t c = d0 + warp * 32; c < d1; c += MG_WARPS * 32) {
            const int32_t i = c + lane;
            int32_t id = -1;
            float v = 0.0f;
            if (i < d1) {
                id = (int32_t)__ldg(u.dir_id16 + i);
                v = __ldg(u.cur + __ldg(u.dir_u + i));
            }
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const float y = __shfl_up_sync(0xffffffffu, v, d);
                const int32_t yid = __shfl_up_sync(0xffffffffu, id, d);
                if (lane >= d && yid == id) v += y;
            }
            const int32_t nid = __shfl_down_sync(0xffffffffu, id, 1);
            if (id >= 0 && (lane == 31 || nid != id)) mine[id] += v;
            __syncwarp();
        }
    }
    __syncthreads();
    const float spread = spread_of(u);
    float dsum = 0.0f;
    for (int t = tid; t < width; t += MG_THREADS) {
        const int32_t v = vbase + t;
        if (v >= u.V) break;
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < MG_WARPS; ++w) sum += acc[(size_t)w * k + t];
        dsum += apply_update(u, v, sum, spread);
    }
    // vertices without any edge (renumbered, from ni on): see k_pull_merge_atomic
    const float r_iso = u.base + u.damping * (0.0f + spread);
    if (u.rank_out)
        for (int64_t v = (int64_t)u.ni + (int64_t)blockIdx.x * MG_THREADS + tid; v < u.V;
             v += (int64_t)gridDim.x * MG_THREADS)
            u.rank_out[u.perm ? __ldg(u.perm + v) : v] = r_iso;
    const float bs = block_sum<float>(dsum, fred);
    grid_sum_last_cta((double)bs, u.dpart, u.counter, u.D_next, (double)(u.V - u.ni) * (double)r_iso);
}

// Rounding to an integer by adding 1.5 * 2^23: for |y| <= 2^22 the sum's low significand
// bits hold round(y) (to nearest, ties to even), and its bit pattern minus that of
// 1.5 * 2^23 is round(y) as an integer.  FP32 adds only: no conversion instruction and no
// FP64 (both slow on GB300).
constexpr float kRndMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int32_t kRndBits = 0x4B400000;  // its bit pattern

// Two-part exact fixed point of xs (an FP32 value scaled by a power of two, |xs| <= 2^44):
// v = hi * 2^22 + lo = round(xs), |hi| <= 2^22, |lo| <= 2^21.  The remainder
// xs - round(xs * 2^-22) * 2^22 is a multiple of the ulp of xs no larger than 2^21, so the FMA
// that forms it is exact; only the last step rounds.  With fewer than 1024 entries per
// vertex neither 32-bit sum can overflow.
__device__ __forceinline__ void fx_split2(float xs, int32_t &hi, int32_t &lo) {
    const float fh = fmaf(xs, 0x1p-22f, kRndMagic);
    hi = __float_as_int(fh) - kRndBits;
    const float r = fmaf(-(fh - kRndMagic), 0x1p22f, xs);
    lo = __float_as_int(r + kRndMagic) - kRndBits;
}

// Three-part form for up to 65535 entries per vertex (|xs| <= 2^48):
// v = hi * 2^32 + mid * 2^16 + lo = round(xs), |hi| <= 2^16, |mid|, |lo| <= 2^15.
__device__ __forceinline__ void fx_split3(float xs, int32_t &hi, int32_t &mid, int32_t &lo) {
    const float fh = fmaf(xs, 0x1p-32f, kRndMagic);
    hi = __float_as_int(fh) - kRndBits;
    const float r1 = fmaf(-(fh - kRndMagic), 0x1p32f, xs);
    const float fm = fmaf(r1, 0x1p-16f, kRndMagic);
    mid = __float_as_int(fm) - kRndBits;
    const float r2 = fmaf(-(fm - kRndMagic), 0x1p16f, r1);
    lo = __float_as_int(r2 + kRndMagic) - kRndBits;
}

// Same slices as k_pull_merge_ordered, one shared accumulator per CTA updated with
// shared-memory atomics, and the slices cut into aligned granules of 8 partials (two 16-byte
// loads of sums and one of 2-byte ids; a granule may reach into the neighbouring ranges'
// entries, which are masked).  The CTA's granules are numbered slice after slice
// and grouped in chunks of 32; warp w takes the w-th sixteenth of the chunks, in order, lane l
// granule l of each, MG_GUNROLL chunks at a time.  The lane finds its first granule's slice
// from a chunk-to-slice map in shared memory (binary search for chunks beyond the map) and the
// following ones by a forward scan.
// MODE 2 / 3: each partial becomes the fixed-point integer of fx_split2 (scale 2^44 per unit
// of mass, fewer than 1024 blocks) or fx_split3 (2^48, fewer than 65536 blocks); the parts
// are added with 32-bit shared reductions and recombined exactly, so the result does not
// depend on the order of the additions: deterministic.  (FP32 shared atomics measured about
// 3.4x slower than 32-bit integer ones on GB300, and 64-bit ones 6.5x.)
constexpr int MG_GRAN = MERGE_GRAN;  // entries per granule: 32 bytes of sums, 16 bytes of 2-byte ids
constexpr int MG_GUNROLL = 2;  // granules of a lane in flight

// Shared-memory layout of k_pull_merge_atomic: nacc accumulator arrays of [k], slice bounds
// and granule prefix ([3B + 1] ints), then (16-byte aligned) the out-degree reciprocals of the
// range's vertices ([k] floats, one bulk copy).
__host__ __device__ inline size_t merge_atomic_inv_offset(int32_t k, int32_t B, int nacc) {
    const size_t head = (size_t)k * 4 * nacc + ((size_t)3 * B + 2) * 4;
    return (head + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t merge_atomic_layout_bytes(int32_t k, int32_t B, int nacc) {
    return merge_atomic_inv_offset(k, B, nacc) + (size_t)k * 4;
}

// Persistent: CTA c reduces range c first, then draws further ranges from a work queue (an
// atomic counter) until none is left.  While one range is reduced, the slice bounds of the
// CTA's next range are already loading (one per thread when B fits the CTA) and the out-degree
// reciprocals of the current range arrive by a bulk copy.  Each range's dangling mass goes to
// its own slot u.dpart[j]; the last CTA adds the slots in range order, so the result does not
// depend on which CTA took which range.
template <int MODE>
__global__ void __launch_bounds__(MG_THREADS, 2) k_pull_merge_atomic(const float *__restrict__ partial,
                                                                     const int32_t *__restrict__ id_map,
                                                                     const uint16_t *__restrict__ id16,
                                                                     const int32_t *__restrict__ offT,
                                                                     const int32_t *__restrict__ gpre_tab, int32_t B,
                                                                     int32_t k, const int32_t *__restrict__ rstart,
                                                                     int32_t nranges, UpdateArgs u) {
    static_assert(MODE == 2 || MODE == 3, "two- or three-part fixed point");
    constexpr int NACC = MODE;
    // launched programmatically after the gather, whose partial sums it reads
    pdl_trigger();
    pdl_wait();
    extern __shared__ __align__(16) unsigned char msm[];
    int32_t *acc_hi = reinterpret_cast<int32_t *>(msm);  // fixed point: NACC arrays of [k]
    int32_t *acc_mid = acc_hi + k;                       // MODE 3 only
    int32_t *acc_lo = acc_hi + (size_t)(NACC - 1) * k;
    int32_t *e_lo = reinterpret_cast<int32_t *>(msm + (size_t)k * 4 * NACC);  // [B] first entry
    int32_t *e_hi = e_lo + B;                                                  // [B] end entry
    int32_t *gpre = e_hi + B;                                                  // [B + 1] granule prefix
    float *sinv = reinterpret_cast<float *>(msm + merge_atomic_inv_offset(k, B, NACC));  // [k]
    __shared__ __align__(8) uint64_t inv_bar;
    __shared__ float wdang[MG_WARPS];  // per-warp dangling mass of the range just finished
    __shared__ int32_t s_next;         // the CTA's next range, drawn from the queue
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // u.fx_scale = 2^61 / mass (a power of two); the parts want 2^44 or 2^48 per unit of mass
    const float scalef = MODE == 2 ? (float)(*u.fx_scale * 0x1p-17) : (float)(*u.fx_scale * 0x1p-13);
    const float inv_scalef = 1.0f / scalef;  // a power of two
    const float spread = spread_of(u);
    const bool one = B < MG_THREADS;  // a thread per block (and one for the total): bounds kept in registers
    if (tid == 0) {
        mbar_init(&inv_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;    // parity of the reciprocal copy's next completion
    bool broken = false;   // a bounded wait gave up: no more copies, ranges skipped
    int32_t j = blockIdx.x, jprev = -1;
    // slice bounds and granule prefix of block tid in range j (when `one`), loaded a range ahead
    int32_t pre_lo = 0, pre_hi = 0, pre_g = 0;
    if (one && tid <= B && j < nranges) {
        if (tid < B) {
            pre_lo = __ldg(offT + (int64_t)j * B + tid);
            pre_hi = __ldg(offT + (int64_t)(j + 1) * B + tid);
        }
        pre_g = __ldg(gpre_tab + (int64_t)j * (B + 1) + tid);
    }
    while (j < nranges) {
        // range j: [j k, (j+1) k), or [rstart[j], rstart[j+1]) (at most k wide) when given
        const int32_t vbase = rstart ? rstart[j] : j * k;
        const int32_t width = rstart ? rstart[j + 1] - vbase : k;
        const int32_t nload = broken ? 0 : min(width, max(0, u.nz - vbase));
        __syncthreads();  // the previous range is done with the accumulators, tables and sinv
        if (tid == 0) {
            if (jprev >= 0) {  // the previous range's dangling mass, warps added in order
                float d = 0.0f;
                for (int w = 0; w < MG_WARPS; ++w) d += wdang[w];
                u.dpart[jprev] = (double)d;
            }
            s_next = (int32_t)gridDim.x + (int32_t)atomicAdd(u.queue, 1u);
        }
        // only the range's own slots are cleared (masked entries add zero to slots < 32, which
        // are never read when the range is narrower)
        for (int a = 0; a < NACC; ++a)
            for (int t = tid; t < width; t += MG_THREADS) acc_hi[(size_t)a * k + t] = 0;
        // the reciprocals of the range's vertices with out-edges arrive by one bulk copy while the
        // partial sums are reduced (vbase is a multiple of 32 and the arrays are padded, so the
        // 16-byte rounded copy stays in bounds)
        if (tid == 0 && nload > 0) {
            const uint32_t bytes = (uint32_t)(nload * 4 + 15) & ~15u;
            mbar_expect_tx(&inv_bar, bytes);
            for (uint32_t off = 0; off < bytes; off += 16384) {
                const uint32_t part = (bytes - off) < 16384u ? (bytes - off) : 16384u;
                bulk_g2s(reinterpret_cast<unsigned char *>(sinv) + off,
                         reinterpret_cast<const unsigned char *>(u.inv_outdeg + vbase) + off, part, &inv_bar);
            }
        }
        // the range's slice bounds and granule prefix (precomputed with the partition) go to
        // shared memory; once the barrier has published the next range's index, its bounds start
        // loading
        if (one) {
            if (tid < B) {
                e_lo[tid] = pre_lo;
                e_hi[tid] = pre_hi;
            }
            if (tid <= B) gpre[tid] = pre_g;
        } else {
            for (int32_t b = tid; b <= B; b += MG_THREADS) {
                if (b < B) {
                    e_lo[b] = __ldg(offT + (int64_t)j * B + b);
                    e_hi[b] = __ldg(offT + (int64_t)(j + 1) * B + b);
                }
                gpre[b] = __ldg(gpre_tab + (int64_t)j * (B + 1) + b);
            }
        }
        __syncthreads();
        const int32_t jn = s_next;
        if (one && tid <= B && jn < nranges) {
            if (tid < B) {
                pre_lo = __ldg(offT + (int64_t)jn * B + tid);
                pre_hi = __ldg(offT + (int64_t)(jn + 1) * B + tid);
            }
            pre_g = __ldg(gpre_tab + (int64_t)jn * (B + 1) + tid);
        }
        const int32_t ngran = gpre[B];
        const int32_t nchunks = (ngran + 31) >> 5;
        const int32_t dummy = lane < k ? lane : 0;  // target of the zero adds of masked entries
        const int32_t c_begin = (int32_t)((int64_t)nchunks * warp / MG_WARPS);
        const int32_t c_end = (int32_t)((int64_t)nchunks * (warp + 1) / MG_WARPS);
        int32_t bp = 0;
        if (c_begin < c_end) {  // the last slice with gpre <= the warp's first granule
            int32_t lo = 0, hi = B - 1;
            const int32_t gq = c_begin << 5;
            while (lo < hi) {
                const int32_t mid = (lo + hi + 1) >> 1;
                if (gpre[mid] <= gq) lo = mid; else hi = mid - 1;
            }
            bp = lo;
        }
        // MG_GUNROLL chunks at a time: all their granule loads are issued before any is added in.
        for (int32_t c0 = c_begin; c0 < c_end; c0 += MG_GUNROLL) {
            float4 xa[MG_GUNROLL], xb[MG_GUNROLL];
            uint4 iv[MG_GUNROLL];
            uint32_t valid[MG_GUNROLL];  // bit e: entry first + e belongs to the slice
#pragma unroll
            for (int q = 0; q < MG_GUNROLL; ++q) {
                const int32_t c = c0 + q;
                const int32_t g = (c << 5) + lane;
                valid[q] = 0u;
                xa[q] = xb[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                iv[q] = make_uint4(0u, 0u, 0u, 0u);
                if (c < c_end && g < ngran) {
                    while (gpre[bp + 1] <= g) ++bp;
                    const int32_t l0 = e_lo[bp], l1 = e_hi[bp];
                    const int32_t f = ((l0 >> 3) + (g - gpre[bp])) << 3;  // MG_GRAN = 8, l0 >= 0
                    const int32_t a = l0 - f > 0 ? l0 - f : 0;              // first valid offset
                    const int32_t z = l1 - f < MG_GRAN ? l1 - f : MG_GRAN;  // end offset
                    valid[q] = (0xFFu >> (MG_GRAN - z)) & (0xFFu << a);
                    // partial sums and ids are read once: streaming loads (evict-first in L2)
                    const float4 *px = reinterpret_cast<const float4 *>(partial + f);
                    xa[q] = __ldcs(px);
                    xb[q] = __ldcs(px + 1);
                    if (id16) {
                        iv[q] = __ldcs(reinterpret_cast<const uint4 *>(id16 + f));
                    } else {  // global ids: keep the granule's position, read them below
                        iv[q].x = (uint32_t)f;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < MG_GUNROLL; ++q) {
                const float x8[MG_GRAN] = {xa[q].x, xa[q].y, xa[q].z, xa[q].w, xb[q].x, xb[q].y, xb[q].z, xb[q].w};
                int32_t id8[MG_GRAN];
                if (id16) {
                    const uint32_t w[4] = {iv[q].x, iv[q].y, iv[q].z, iv[q].w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        id8[2 * h] = (int32_t)(w[h] & 0xFFFFu);
                        id8[2 * h + 1] = (int32_t)(w[h] >> 16);
                    }
                } else {
                    int4 w0 = make_int4(vbase, vbase, vbase, vbase), w1 = w0;
                    if (valid[q]) {
                        const int4 *pi = reinterpret_cast<const int4 *>(id_map + (int32_t)iv[q].x);
                        w0 = __ldg(pi);
                        w1 = __ldg(pi + 1);
                    }
                    id8[0] = w0.x - vbase; id8[1] = w0.y - vbase; id8[2] = w0.z - vbase; id8[3] = w0.w - vbase;
                    id8[4] = w1.x - vbase; id8[5] = w1.y - vbase; id8[6] = w1.z - vbase; id8[7] = w1.w - vbase;
                }
                // Entries outside the slice add zero to a slot of their own lane (no branches: the
                // atomics of a warp stay converged; predicating them off measured slower).
#pragma unroll
                for (int e = 0; e < MG_GRAN; ++e) {
                    const bool ok = (valid[q] >> e) & 1u;
                    const int32_t id = ok ? id8[e] : dummy;
                    const float x = ok ? x8[e] : 0.0f;
                    if (MODE == 2) {
                        int32_t h, lw;
                        fx_split2(x * scalef, h, lw);
                        atomicAdd(acc_hi + id, h);
                        atomicAdd(acc_lo + id, lw);
                    } else {
                        int32_t h, md, lw;
                        fx_split3(x * scalef, h, md, lw);
                        if (h) atomicAdd(acc_hi + id, h);
                        atomicAdd(acc_mid + id, md);
                        atomicAdd(acc_lo + id, lw);
                    }
                }
            }
        }
        if (u.dir_off) {  // the range's direct pieces: their sources' contributions, read here
            const int32_t d0 = __ldg(u.dir_off + j), d1 = __ldg(u.dir_off + j + 1);
            const int32_t f0 = d0 & ~(MG_GRAN - 1);
            const int32_t ng = d1 > d0 ? (d1 - f0 + MG_GRAN - 1) / MG_GRAN : 0;
            for (int32_t gi = tid; gi < ng; gi += MG_THREADS) {
                const int32_t f = f0 + gi * MG_GRAN;
                const int32_t a = d0 - f > 0 ? d0 - f : 0;              // first valid offset
                const int32_t z = d1 - f < MG_GRAN ? d1 - f : MG_GRAN;  // end offset
                const uint32_t valid = (0xFFu >> (MG_GRAN - z)) & (0xFFu << a);
                const int4 s0 = __ldg(reinterpret_cast<const int4 *>(u.dir_u + f));
                const int4 s1 = __ldg(reinterpret_cast<const int4 *>(u.dir_u + f) + 1);
                const uint4 iv = __ldg(reinterpret_cast<const uint4 *>(u.dir_id16 + f));
                const int32_t src[MG_GRAN] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
                float x8[MG_GRAN];
#pragma unroll
                for (int e = 0; e < MG_GRAN; ++e) x8[e] = ((valid >> e) & 1u) ? __ldg(u.cur + src[e]) : 0.0f;
                const uint32_t w[4] = {iv.x, iv.y, iv.z, iv.w};
#pragma unroll
                for (int e = 0; e < MG_GRAN; ++e) {
                    const bool ok = (valid >> e) & 1u;
                    const int32_t id = ok ? (int32_t)((w[e >> 1] >> (16 * (e & 1))) & 0xFFFFu) : dummy;
                    const float x = ok ? x8[e] : 0.0f;
                    if (MODE == 2) {
                        int32_t h, lw;
                        fx_split2(x * scalef, h, lw);
                        atomicAdd(acc_hi + id, h);
                        atomicAdd(acc_lo + id, lw);
                    } else {
                        int32_t h, md, lw;
                        fx_split3(x * scalef, h, md, lw);
                        if (h) atomicAdd(acc_hi + id, h);
                        atomicAdd(acc_mid + id, md);
                        atomicAdd(acc_lo + id, lw);
                    }
                }
            }
        }
        __syncthreads();
        // bounded wait for the reciprocals; on a timeout the flag is set (the caller reports
        // TC_ERR_TIMEOUT) and this and every later range of the CTA are skipped, but the CTA
        // still joins the dangling-mass reduction so that its arrival counter stays consistent
        if (nload > 0) {
            if (!mbar_wait(&inv_bar, phase, u.err, 2)) broken = true;
            phase ^= 1u;
        }
        float dsum = 0.0f;
        for (int t = tid; !broken && t < width; t += MG_THREADS) {
            const int32_t v = vbase + t;
            if (v >= u.V) break;
            // exact 64-bit total, converted with 32-bit integer-to-float steps (no FP64)
            const long long tot = MODE == 2 ? ((long long)acc_hi[t] << 22) + (long long)acc_lo[t]
                                            : ((long long)acc_hi[t] << 32) + ((long long)acc_mid[t] << 16) +
                                                  (long long)acc_lo[t];
            const float th = (float)(int32_t)(tot >> 24);            // |tot| < 2^49
            const float tl = (float)(uint32_t)(tot & 0xFFFFFFll);     // < 2^24, exact
            const float sum = fmaf(th, 16777216.0f, tl) * inv_scalef;
            dsum += apply_update_inv(u, v, sum, spread, t < nload ? sinv[t] : 0.0f);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, d);
        if (lane == 0) wdang[warp] = dsum;
        jprev = j;
        j = jn;
    }
    __syncthreads();
    if (tid == 0 && jprev >= 0) {
        float d = 0.0f;
        for (int w = 0; w < MG_WARPS; ++w) d += wdang[w];
        u.dpart[jprev] = (double)d;
    }
    // Vertices without any edge (renumbered to the end, from ni on) get no pieces and pass nothing
    // on: every one of them has the rank of an empty sum, and their dangling mass is that rank
    // times their count, added once by the last CTA.
    const float r_iso = u.base + u.damping * (0.0f + spread);
    if (u.rank_out)
        for (int64_t v = (int64_t)u.ni + (int64_t)blockIdx.x * MG_THREADS + tid; v < u.V;
             v += (int64_t)gridDim.x * MG_THREADS)
            u.rank_out[u.perm ? __ldg(u.perm + v) : v] = r_iso;
    grid_sum_slots_last_cta(u.dpart, nranges, u.counter, u.queue, u.D_next, (double)(u.V - u.ni) * (double)r_iso);
}

// Entries per vertex are at most B (one per block): two-part fixed point below 1024 blocks.
int merge_fixed_parts(int32_t B) { return B < 1024 ? 2 : 3; }

size_t merge_atomic_smem_bytes(int32_t k, int32_t B, bool fixed) {
    return merge_atomic_layout_bytes(k, B, fixed ? merge_fixed_parts(B) : 1);
}

// Initial ranks (1/V or caller's), first contributions, their dangling mass, and the
// fixed-point scale of the merge: 2^61 / max(1, sum |r|).  No later iteration has a larger
// L1 mass (each is (1-d) + d * previous at most), so no vertex sum can overflow 2^63.
__global__ void __launch_bounds__(PR_THREADS) k_pr_init(const float *__restrict__ init, UpdateArgs u, double *mass,
                                                         double *scale) {
    pdl_wait();  // launched programmatically after the previous call's last kernel
    __shared__ float fred[32];
    float dsum = 0.0f, msum = 0.0f;
    const float r0 = 1.0f / (float)u.V;
    for (int64_t v = blockIdx.x * (int64_t)PR_THREADS + threadIdx.x; v < u.V; v += (int64_t)gridDim.x * PR_THREADS) {
        const int32_t orig = u.perm ? __ldg(u.perm + v) : (int32_t)v;  // caller's ID of vertex v
        const float r = init ? init[orig] : r0;
        if (u.rank_out) u.rank_out[orig] = r;
        const float inv = __ldg(u.inv_outdeg + v);
        u.contrib_next[v] = r * inv;
        if (inv == 0.0f) dsum += r;
        msum += fabsf(r);
    }
    const float bs = block_sum<float>(dsum, fred);
    const float bm = block_sum<float>(msum, fred);
    if (grid_sum2_last_cta((double)bs, (double)bm, u.dpart, u.counter, u.D_next, mass) && threadIdx.x == 0) {
        // 2^61 / 2^ceil(log2(max(1, mass))): a power of two (so FP32 values scale exactly), and
        // a vertex sum is at most the mass, so |sum * scale| <= 2^61 < 2^63.
        const double m = *mass;
        int e = 0;
        if (m > 1.0) e = (int)ceil(log2(m));
        *scale = ldexp(1.0, 61 - e);
    }
}


// ---------------------------------------------------------------------------------------------
// Push scatter (Alg. 2; Alg. 5 when id_map != null): every edge s -> d adds contrib[s] to
// sums[d] by a reduction in L2.  FIXED: 64-bit fixed-point integer reductions (red.add.u64),
// exact in any order, so the ranks repeat bit for bit; otherwise FP32 atomicAdd (the paper's
// form, order-dependent rounding).
// ---------------------------------------------------------------------------------------------

// round(y) as a 64-bit two's-complement integer for |y| < 2^62, from the FP32 bits (integer
// operations only: 64-bit float-to-integer conversions run on the FP64 unit).
__device__ __forceinline__ unsigned long long fx_round64(float y) {
    const uint32_t b = __float_as_uint(y);
    const uint32_t a = b & 0x7fffffffu;
    const int e = (int)(a >> 23);
    const unsigned long long m = (a & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = (e ? e : 1) - 150;  // |y| = m * 2^sh
    unsigned long long r;
    if (sh >= 0) r = m << sh;
    else if (sh <= -25) r = 0ull;
    else r = (m + (1ull << (-sh - 1))) >> (-sh);  // to nearest, ties away from zero
    return (b >> 31) ? (0ull - r) : r;
}

template <bool FIXED>
__device__ __forceinline__ void push_add(void *sums, int32_t d, float c, float scalef) {
    if (FIXED) atomicAdd(static_cast<unsigned long long *>(sums) + d, fx_round64(c * scalef));
    else atomicAdd(static_cast<float *>(sums) + d, c);
}

// The push sums' fixed-point scale: 2^55 per unit of the largest L1 mass, so that |sum| < 2^55
// (the update converts it with 32-bit steps).
__device__ __forceinline__ float push_scale(const double *fx_scale) { return (float)(*fx_scale * 0x1p-6); }

// Thread/warp/CTA mapping of the rows (Sec. 3.2's TWC): short rows a lane each, rows of at least
// warp_min edges a warp each, hubs a CTA each.
template <bool FIXED>
__global__ void __launch_bounds__(PR_THREADS) k_push_scatter(const int32_t *__restrict__ rowptr,
                                                             const int32_t *__restrict__ colidx, int64_t nrows,
                                                             const int32_t *__restrict__ id_map,
                                                             const int32_t *__restrict__ hubs, int32_t num_hubs,
                                                             int32_t hub_degree, int hub_ctas,
                                                             const float *__restrict__ contrib, void *sums,
                                                             const double *fx_scale, LbArgs lb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float scalef = FIXED ? push_scale(fx_scale) : 1.0f;
    if ((int)blockIdx.x < hub_ctas) {
        for (int32_t h = blockIdx.x; h < num_hubs; h += hub_ctas) {
            const int32_t row = hubs[h];
            const int32_t src = id_map ? __ldg(id_map + row) : row;
            const float c = __ldg(contrib + src);
            const int32_t s = rowptr[row], e = rowptr[row + 1];
            if (c != 0.0f)
                for (int32_t i = s + threadIdx.x; i < e; i += PR_THREADS) push_add<FIXED>(sums, __ldg(colidx + i), c, scalef);
        }
        return;
    }
    const int64_t ngroups = (nrows + 31) >> 5;
    const int64_t nwarps = (int64_t)(gridDim.x - hub_ctas) * PR_WARPS;
    for (int64_t grp = (int64_t)(blockIdx.x - hub_ctas) * PR_WARPS + warp; grp < ngroups; grp += nwarps) {
        const int64_t row = grp * 32 + lane;
        const bool valid = row < nrows;
        int32_t s = 0, e = 0;
        float c = 0.0f;
        if (valid) {
            s = __ldg(rowptr + row);
            e = __ldg(rowptr + row + 1);
            c = __ldg(contrib + (id_map ? __ldg(id_map + row) : (int32_t)row));
        }
        const int32_t deg = e - s;
        const int32_t wmin = lb_warp_min(lb, grp * 32);
        if (deg < wmin && deg <= hub_degree && c != 0.0f)  // hubs are scattered by their CTA only
            for (int32_t i = s; i < e; ++i) push_add<FIXED>(sums, __ldg(colidx + i), c, scalef);
        unsigned wm = __ballot_sync(0xffffffffu, valid && deg >= wmin && deg <= hub_degree && c != 0.0f);
        while (wm) {
            const int l = __ffs(wm) - 1;
            wm &= wm - 1;
            const int32_t ws = __shfl_sync(0xffffffffu, s, l), we = __shfl_sync(0xffffffffu, e, l);
            const float cl = __shfl_sync(0xffffffffu, c, l);
            for (int32_t i = ws + lane; i < we; i += 32) push_add<FIXED>(sums, __ldg(colidx + i), cl, scalef);
        }
    }
}

// Edge-parallel mapping: thread t takes edges t, t + T, ... of the whole stream (every edge the
// same work, so no row is a straggler).  esrc[i] is the source of edge i; consecutive edges
// share it, so its contribution mostly comes from L1.  The grid walks the edges in order, so
// with a partition the blocks - and their L2-resident destination ranges - pass one by one.
template <bool FIXED>
__global__ void __launch_bounds__(PR_THREADS) k_push_edges(const int32_t *__restrict__ esrc,
                                                           const int32_t *__restrict__ dst, int64_t E,
                                                           const float *__restrict__ contrib, void *sums,
                                                           const double *fx_scale) {
    const float scalef = FIXED ? push_scale(fx_scale) : 1.0f;
    const int64_t T = (int64_t)gridDim.x * PR_THREADS;
    int64_t i = blockIdx.x * (int64_t)PR_THREADS + threadIdx.x;
    for (; i + 3 * T < E; i += 4 * T) {  // four edges in flight per thread
        int32_t sv[4], dv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sv[k] = __ldg(esrc + i + k * T);
            dv[k] = __ldg(dst + i + k * T);
        }
        float cv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[k] = __ldg(contrib + sv[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (cv[k] != 0.0f) push_add<FIXED>(sums, dv[k], cv[k], scalef);
    }
    for (; i < E; i += T) {
        const float c = __ldg(contrib + __ldg(esrc + i));
        if (c != 0.0f) push_add<FIXED>(sums, __ldg(dst + i), c, scalef);
    }
}

template <bool FIXED>
__global__ void __launch_bounds__(PR_THREADS) k_push_update(void *sums, UpdateArgs u) {
    __shared__ float fred[32];
    const float spread = spread_of(u);
    const float inv_scalef = FIXED ? 1.0f / push_scale(u.fx_scale) : 1.0f;  // a power of two
    float dsum = 0.0f;
    for (int64_t v = blockIdx.x * (int64_t)PR_THREADS + threadIdx.x; v < u.V; v += (int64_t)gridDim.x * PR_THREADS) {
        float s;
        if (FIXED) {
            unsigned long long *sp = static_cast<unsigned long long *>(sums) + v;
            const long long tot = (long long)*sp;
            *sp = 0ull;
            const float th = (float)(int32_t)(tot >> 24);          // |tot| < 2^55
            const float tl = (float)(uint32_t)(tot & 0xFFFFFFll);  // < 2^24, exact
            s = fmaf(th, 16777216.0f, tl) * inv_scalef;
        } else {
            float *sp = static_cast<float *>(sums) + v;
            s = *sp;
            *sp = 0.0f;
        }
        dsum += apply_update(u, (int32_t)v, s, spread);
    }
    const float bs = block_sum<float>(dsum, fred);
    grid_sum_last_cta((double)bs, u.dpart, u.counter, u.D_next);
}

// ---------------------------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------------------------
struct Timer {
    bool on = false;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    float *acc = nullptr;
    int begin(bool enable, cudaStream_t st, float *target) {
        on = enable;
        s = st;
        acc = target;
        if (!on) return TC_OK;
        TC_CUDA(cudaEventCreate(&ev[0]));
        TC_CUDA(cudaEventCreate(&ev[1]));
        TC_CUDA(cudaEventRecord(ev[0], s));
        return TC_OK;
    }
    int end() {
        if (!on) return TC_OK;
        TC_CUDA(cudaEventRecord(ev[1], s));
        TC_CUDA(cudaEventSynchronize(ev[1]));
        float ms = 0;
        TC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        *acc += ms;
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
        return TC_OK;
    }
};

static int occupancy_grid(const void *kernel, int threads, size_t smem, int64_t work_ctas, int *grid) {
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    int per_sm = 0;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) per_sm = 1;
    int64_t g = (int64_t)caps.sms * per_sm;
    if (work_ctas < g) g = work_ctas;
    if (g < 1) g = 1;
    *grid = (int)g;
    return TC_OK;
}

struct PrState {
    float *contrib[2];
    double *D;          // D[0], D[1]
    unsigned *counter;
    unsigned *queue;    // work queue of the persistent merge
    double *mass;       // L1 mass of the initial ranks
    double *scale;      // fixed-point scale of the merge
    int *err;           // sticky error flag of bounded device waits
    double *dpart;      // per-CTA partials (capacity 2 * dpart_cap doubles)
    int64_t dpart_cap;
    float *rank_dev;    // ranks on the device (caller's buffer or scratch)
    float *sums;        // push only
};

static int prepare_state(tc_graph *g, const tc_pr_params *pp, float *ranks_out, bool push, int64_t max_ctas,
                         PrState *st) {
    const int32_t V = g->V;
    const int64_t Vp = ((int64_t)V + 63) / 64 * 64;  // 256-byte aligned vectors, padded for bulk copies
    TC_TRY(g->ws_contrib.alloc((size_t)Vp * 4 * (push ? 4 : 2) + 256));  // push: 8-byte sums
    st->contrib[0] = g->ws_contrib.as<float>();
    st->contrib[1] = st->contrib[0] + Vp;
    st->sums = push ? st->contrib[1] + Vp : nullptr;
    st->dpart_cap = max_ctas;
    const bool fresh = g->ws_scalars.p == nullptr;
    TC_TRY(g->ws_scalars.alloc(128 + (size_t)max_ctas * 16));
    char *sc = g->ws_scalars.as<char>();
    st->D = reinterpret_cast<double *>(sc);
    st->counter = reinterpret_cast<unsigned *>(sc + 32);
    st->queue = reinterpret_cast<unsigned *>(sc + 36);
    st->err = reinterpret_cast<int *>(sc + 40);
    st->mass = reinterpret_cast<double *>(sc + 48);
    st->scale = reinterpret_cast<double *>(sc + 56);
    st->dpart = reinterpret_cast<double *>(sc + 128);
    (void)fresh;
    if (pp->out_mem == TC_MEM_DEVICE) {
        st->rank_dev = ranks_out;
    } else {
        TC_TRY(g->ws_misc.alloc((size_t)V * 4 + 256));
        st->rank_dev = g->ws_misc.as<float>();
    }
    return TC_OK;
}

static int check_pr_args(const tc_graph *g, const tc_part *part, const tc_pr_params *pp, float *ranks_out, int dir) {
    if (!g || !pp || !ranks_out) return fail(TC_ERR_INVALID_ARG, "pagerank: null graph, params or output");
    if (!(pp->damping >= 0.0f && pp->damping <= 1.0f)) return fail(TC_ERR_INVALID_ARG, "pagerank: damping outside [0,1]");
    if (pp->iters < 0) return fail(TC_ERR_INVALID_ARG, "pagerank: iters < 0");
    if (pp->dangling != TC_DANGLING_REDISTRIBUTE && pp->dangling != TC_DANGLING_DROP)
        return fail(TC_ERR_INVALID_ARG, "pagerank: bad dangling mode");
    if (pp->out_mem != TC_MEM_HOST && pp->out_mem != TC_MEM_DEVICE)
        return fail(TC_ERR_INVALID_ARG, "pagerank: bad out_mem");
    if (pp->lb_warp_min < 0) return fail(TC_ERR_INVALID_ARG, "pagerank: lb_warp_min < 0");
    if (pp->merge_mode != TC_MERGE_FIXED && pp->merge_mode != TC_MERGE_ORDERED &&
        !(dir == TC_PUSH && pp->merge_mode == TC_PUSH_FLOAT))
        return fail(TC_ERR_INVALID_ARG, "pagerank: bad merge_mode");
    if (part && (part->g != g || part->dir != dir))
        return fail(TC_ERR_INVALID_ARG, "pagerank: partition belongs to another graph or direction");
    return TC_OK;
}

// The source of every out-edge of the graph (its row in the out-CSR), built on first use by the
// edge-parallel push and kept with the graph.
static int push_sources(tc_graph *g, cudaStream_t s) {
    if (g->push_esrc_built) return TC_OK;
    TC_TRY(g->push_esrc.alloc((size_t)(g->E > 0 ? g->E : 1) * 4));
    if (g->E > 0) TC_TRY(expand_rows(g->out_rowptr.as<int32_t>(), g->V, g->push_esrc.as<int32_t>(), s));
    TC_CUDA(cudaStreamSynchronize(s));
    g->push_esrc_built = true;
    return TC_OK;
}

static int pagerank_impl(const tc_graph *cg, const tc_part *part, const tc_pr_params *pp, float *ranks_out,
                         tc_pr_stats *stats, cudaStream_t s, bool push) {
    tc_graph *g = const_cast<tc_graph *>(cg);  // scratch buffers only
    const int32_t V = g->V;
    if (stats) memset(stats, 0, sizeof(*stats));
    if (V == 0) return TC_OK;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));

    // launch shapes
    int g_gather = 1, g_upd = 1, g_merge = 1, hub_ctas = 0;
    int64_t nrows;
    int64_t max_ctas_hint = 1;
    const int32_t *rp, *ci, *hubs, *idm = nullptr;
    int32_t nhubs, hubdeg;
    if (part) {
        nrows = part->R;
        rp = part->rowptr.as<int32_t>();
        ci = part->colidx.as<int32_t>();
        hubs = part->hubs.as<int32_t>();
        nhubs = part->num_hubs;
        hubdeg = part->hub_degree;
        idm = part->id_map.as<int32_t>();
    } else {
        nrows = V;
        rp = push ? g->out_rowptr.as<int32_t>() : g->in_rowptr.as<int32_t>();
        ci = push ? g->out_colidx.as<int32_t>() : g->in_colidx.as<int32_t>();
        hubs = push ? g->out_hubs.as<int32_t>() : g->in_hubs.as<int32_t>();
        nhubs = push ? g->num_out_hubs : g->num_in_hubs;
        hubdeg = g->hub_degree;
    }
    hub_ctas = nhubs > 0 ? (nhubs < caps.sms ? nhubs : caps.sms) : 0;
    const bool tiled = part && !push && part->tiled;
    const int64_t group_ctas = ((nrows + 31) / 32 + PR_WARPS - 1) / PR_WARPS;
    const void *kgather = push ? (const void *)k_push_scatter<true>
                               : (part ? (const void *)k_pull_gather<false> : (const void *)k_pull_gather<true>);
    TC_TRY(occupancy_grid(kgather, PR_THREADS, 0, group_ctas > 0 ? group_ctas : 1, &g_gather));
    g_gather += hub_ctas;
    TC_TRY(occupancy_grid((const void *)k_push_update<true>, PR_THREADS, 0, ((int64_t)V + PR_THREADS - 1) / PR_THREADS,
                          &g_upd));
    size_t merge_smem = 0;
    int merge_mode = TC_MERGE_FIXED;
    if (part && !push) {
        g_merge = part->nranges;
        merge_mode = pp->merge_mode;
        // per-warp accumulators that do not fit in shared memory: the exact fixed-point merge
        // (also deterministic) takes over
        if (merge_mode == TC_MERGE_ORDERED && merge_smem_bytes(part->k, part->B) > (size_t)caps.max_smem_optin)
            merge_mode = TC_MERGE_FIXED;
        if (merge_mode == TC_MERGE_ORDERED) {
            merge_smem = merge_smem_bytes(part->k, part->B);
            TC_CUDA(cudaFuncSetAttribute(k_pull_merge_ordered, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)merge_smem));
        } else {
            merge_smem = merge_atomic_smem_bytes(part->k, part->B, true);
            const void *kmerge = merge_fixed_parts(part->B) == 2 ? (const void *)k_pull_merge_atomic<2>
                                                                 : (const void *)k_pull_merge_atomic<3>;
            // always: the 48 KB default also counts the kernel's static shared memory
            TC_CUDA(cudaFuncSetAttribute(kmerge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)merge_smem));
            // persistent: as many CTAs as fit on the device at once (each loops over ranges)
            TC_TRY(occupancy_grid(kmerge, MG_THREADS, merge_smem, part->nranges, &g_merge));
        }
    }
    int g_init = 1;
    TC_TRY(occupancy_grid((const void *)k_pr_init, PR_THREADS, 0, ((int64_t)V + PR_THREADS - 1) / PR_THREADS, &g_init));
    int64_t max_ctas = g_gather;
    if (g_init > max_ctas) max_ctas = g_init;
    if (max_ctas_hint > max_ctas) max_ctas = max_ctas_hint;
    if (g_upd > max_ctas) max_ctas = g_upd;
    if (g_merge > max_ctas) max_ctas = g_merge;
    if (part && !push && part->nranges > max_ctas) max_ctas = part->nranges;  // one dangling slot per range

    PrState st;
    TC_TRY(prepare_state(g, pp, ranks_out, push, max_ctas, &st));
    TC_CUDA(cudaMemsetAsync(st.counter, 0, 16, s));  // counter, merge work queue and the error flag
    if (push) TC_CUDA(cudaMemsetAsync(st.sums, 0, (size_t)V * 8, s));
    // push: fixed-point sums unless FP32 atomics are asked for; the edge-parallel scatter unless
    // a TWC warp threshold (lb_warp_min or a per-block table) is given
    const bool push_fixed = pp->merge_mode != TC_PUSH_FLOAT;
    const bool push_staged = push && part && part->nptiles > 0 && pp->lb_warp_min == 0 && !part->lb_tab.p;
    const bool push_edges = push && !push_staged && pp->lb_warp_min == 0 && !(part && part->lb_tab.p);
    const int32_t *esrc = nullptr;
    int64_t nedges = 0;
    int g_edges = 1;
    if (push_edges) {
        if (part) {
            esrc = part->esrc.as<int32_t>();
            nedges = part->E;
        } else {
            TC_TRY(push_sources(g, s));
            esrc = g->push_esrc.as<int32_t>();
            nedges = g->E;
        }
        TC_TRY(occupancy_grid((const void *)k_push_edges<true>, PR_THREADS, 0,
                              (nedges + PR_THREADS - 1) / PR_THREADS > 0 ? (nedges + PR_THREADS - 1) / PR_THREADS : 1,
                              &g_edges));
    }

    UpdateArgs u;
    u.base = (1.0f - pp->damping) / (float)V;
    u.damping = pp->damping;
    u.drop = pp->dangling == TC_DANGLING_DROP;
    u.V = V;
    u.dpart = st.dpart;
    u.counter = st.counter;
    const bool renumbered = part && part->order == TC_ORDER_OUTDEGREE;
    u.inv_outdeg = renumbered ? part->inv_outdeg.as<float>() : g->inv_outdeg.as<float>();
    u.fx_scale = st.scale;
    u.perm = renumbered ? part->perm.as<int32_t>() : nullptr;
    u.nz = renumbered ? part->nz_out : V;
    u.ni = renumbered ? part->ni : V;
    u.err = st.err;
    u.queue = st.queue;
    const bool direct = part && part->ndirect > 0;
    u.dir_off = direct ? part->dir_off.as<int32_t>() : nullptr;
    u.dir_u = direct ? part->dir_u.as<int32_t>() : nullptr;
    u.dir_id16 = direct ? part->dir_id16.as<uint16_t>() : nullptr;
    u.cur = nullptr;

    // the window applies to the unstaged pull gathers (the staged one copies its block's values
    // to shared memory)
    L2Window l2w;
    if (pp->l2_window && !push && !tiled) TC_TRY(l2w.begin((size_t)V * 4, s));

    float ms_total = 0, ms_gather = 0, ms_merge = 0;
    Timer tt;
    TC_TRY(tt.begin(pp->profile != 0, s, &ms_total));
    int launches = 0;
    // init: contributions[0], D[0]
    u.D_cur = st.D + 1;
    u.D_next = st.D + 0;
    u.rank_out = pp->iters == 0 ? st.rank_dev : nullptr;
    u.contrib_next = st.contrib[0];
    {
        const float *init_dev = pp->init;
        if (pp->init && pp->out_mem == TC_MEM_HOST) {
            TC_CUDA(cudaMemcpyAsync(st.rank_dev, pp->init, (size_t)V * 4, cudaMemcpyHostToDevice, s));
            init_dev = st.rank_dev;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g_init);
        cfg.blockDim = dim3(PR_THREADS);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        TC_CUDA(cudaLaunchKernelEx(&cfg, k_pr_init, init_dev, u, st.mass, st.scale));
        launches += 1;
    }
    for (int it = 0; it < pp->iters; ++it) {
        const bool last = it == pp->iters - 1;
        const float *cur = push ? st.contrib[0] : st.contrib[it & 1];
        u.D_cur = st.D + (it & 1);
        u.D_next = st.D + ((it + 1) & 1);
        u.rank_out = last ? st.rank_dev : nullptr;
        u.contrib_next = push ? st.contrib[0] : st.contrib[(it + 1) & 1];
        u.cur = cur;
        Timer t1;
        TC_TRY(t1.begin(pp->profile != 0, s, &ms_gather));
        LbArgs lb;
        lb.warp_min = pp->lb_warp_min > 0 ? pp->lb_warp_min : 32;
        lb.lb_tab = (part && part->lb_tab.p) ? part->lb_tab.as<int32_t>() : nullptr;
        lb.blk_rows = part ? part->blk_rows_dev.as<int64_t>() : nullptr;
        lb.B = part ? part->B : 1;
        if (push) {
            if (push_staged)
                TC_TRY(launch_push_smem(part, cur, st.sums, st.scale, push_fixed, s));
            else if (push_edges && push_fixed)
                k_push_edges<true><<<g_edges, PR_THREADS, 0, s>>>(esrc, ci, nedges, cur, st.sums, st.scale);
            else if (push_edges)
                k_push_edges<false><<<g_edges, PR_THREADS, 0, s>>>(esrc, ci, nedges, cur, st.sums, st.scale);
            else if (push_fixed)
                k_push_scatter<true><<<g_gather, PR_THREADS, 0, s>>>(rp, ci, nrows, idm, hubs, nhubs, hubdeg,
                                                                     hub_ctas, cur, st.sums, st.scale, lb);
            else
                k_push_scatter<false><<<g_gather, PR_THREADS, 0, s>>>(rp, ci, nrows, idm, hubs, nhubs, hubdeg,
                                                                      hub_ctas, cur, st.sums, st.scale, lb);
        } else if (tiled) {
            int nl = 0;
            TC_TRY(launch_tiled_gather(part, cur, st.err, s, &nl));
            launches += nl - 1;
        } else if (l2w.on) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(g_gather);
            cfg.blockDim = dim3(PR_THREADS);
            cfg.stream = s;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
            attr[0].val.accessPolicyWindow = l2w.window(cur, (size_t)V * 4);
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            float *partial = part ? part->partial.as<float>() : nullptr;
            if (part)
                TC_CUDA(cudaLaunchKernelEx(&cfg, k_pull_gather<false>, rp, ci, nrows, hubs, nhubs, hubdeg, hub_ctas,
                                           cur, partial, u, lb));
            else
                TC_CUDA(cudaLaunchKernelEx(&cfg, k_pull_gather<true>, rp, ci, nrows, hubs, nhubs, hubdeg, hub_ctas,
                                           cur, partial, u, lb));
        } else if (part) {
            k_pull_gather<false><<<g_gather, PR_THREADS, 0, s>>>(rp, ci, nrows, hubs, nhubs, hubdeg, hub_ctas, cur,
                                                                 part->partial.as<float>(), u, lb);
        } else {
            k_pull_gather<true><<<g_gather, PR_THREADS, 0, s>>>(rp, ci, nrows, hubs, nhubs, hubdeg, hub_ctas, cur,
                                                                nullptr, u, lb);
        }
        TC_LAUNCH_CHECK();
        ++launches;
        TC_TRY(t1.end());
        if (push || part) {
            Timer t2;
            TC_TRY(t2.begin(pp->profile != 0, s, &ms_merge));
            if (push) {
                if (push_fixed) k_push_update<true><<<g_upd, PR_THREADS, 0, s>>>(st.sums, u);
                else k_push_update<false><<<g_upd, PR_THREADS, 0, s>>>(st.sums, u);
            } else {
                const uint16_t *i16 = part->id16.p ? part->id16.as<uint16_t>() : nullptr;
                const int32_t *rst = part->rstart.p ? part->rstart.as<int32_t>() : nullptr;
                if (merge_mode == TC_MERGE_ORDERED)
                    k_pull_merge_ordered<<<g_merge, MG_THREADS, merge_smem, s>>>(
                        part->partial.as<float>(), part->id_map.as<int32_t>(), i16, part->merge_offT.as<int32_t>(),
                        part->B, part->k, rst, u);
                else {
                    cudaLaunchConfig_t cfg = {};
                    cfg.gridDim = dim3(g_merge);
                    cfg.blockDim = dim3(MG_THREADS);
                    cfg.dynamicSmemBytes = merge_smem;
                    cfg.stream = s;
                    cudaLaunchAttribute attr[1];
                    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                    attr[0].val.programmaticStreamSerializationAllowed = 1;
                    cfg.attrs = attr;
                    cfg.numAttrs = 1;
                    const float *pa = part->partial.as<float>();
                    const int32_t *im = part->id_map.as<int32_t>(), *ot = part->merge_offT.as<int32_t>(),
                                  *gp = part->merge_gpre.as<int32_t>();
                    if (merge_fixed_parts(part->B) == 2)
                        TC_CUDA(cudaLaunchKernelEx(&cfg, k_pull_merge_atomic<2>, pa, im, i16, ot, gp, part->B, part->k,
                                                   rst, part->nranges, u));
                    else
                        TC_CUDA(cudaLaunchKernelEx(&cfg, k_pull_merge_atomic<3>, pa, im, i16, ot, gp, part->B, part->k,
                                                   rst, part->nranges, u));
                }
            }
            TC_LAUNCH_CHECK();
            ++launches;
            TC_TRY(t2.end());
        }
    }
    TC_TRY(tt.end());
    TC_TRY(l2w.end());
    if (pp->out_mem == TC_MEM_HOST)
        TC_CUDA(cudaMemcpyAsync(ranks_out, st.rank_dev, (size_t)V * 4, cudaMemcpyDeviceToHost, s));
    if (stats || pp->out_mem == TC_MEM_HOST) {
        int err = 0;
        TC_CUDA(cudaMemcpyAsync(&err, st.err, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        if (err) return fail(TC_ERR_TIMEOUT, "pagerank: a bounded device wait gave up (code %d)", err);
    }
    if (stats) {
        double D = 0;
        TC_CUDA(cudaMemcpyAsync(&D, st.D + (pp->iters & 1), 8, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        stats->dangling_mass = D;
        stats->iters = pp->iters;
        stats->launches = launches;
        stats->ms_total = ms_total;
        stats->ms_gather = ms_gather;
        stats->ms_merge = ms_merge;
    } else if (pp->out_mem == TC_MEM_HOST) {
        TC_CUDA(cudaStreamSynchronize(s));
    }
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_pagerank_pull(const tc_graph *g, const tc_part *part, const tc_pr_params *params, float *ranks_out,
                                tc_pr_stats *stats, void *stream) {
    TC_TRY(tc::check_pr_args(g, part, params, ranks_out, TC_PULL));
    return tc::pagerank_impl(g, part, params, ranks_out, stats, (cudaStream_t)stream, false);
}

extern "C" int tc_pagerank_push(const tc_graph *g, const tc_part *part, const tc_pr_params *params, float *ranks_out,
                                tc_pr_stats *stats, void *stream) {
    TC_TRY(tc::check_pr_args(g, part, params, ranks_out, TC_PUSH));
    return tc::pagerank_impl(g, part, params, ranks_out, stats, (cudaStream_t)stream, true);
}
