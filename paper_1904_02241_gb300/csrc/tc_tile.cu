// Shared-memory staged TOCAB gather (Alg. 4 with the block's vertex values on chip).
//
// The paper sizes a block so that its contributions fit in the last-level cache (Sec. 3.1).
// On GB300 the whole contribution vector of a scale-24 graph already fits in the 135 MB L2,
// and the random requests themselves become the bound (one L1/L2 sector request per edge).
// This format sizes a block so that its contributions fit in one CTA's shared memory instead,
// where a random warp gather costs a few bank cycles:
//   * a block's contributions are copied into shared memory with bulk asynchronous copies
//     (TMA, cp.async.bulk) completing on an mbarrier;
//   * col16[]  : uint16 source offset inside the block (source - b*W), each block's edges
//                padded to a multiple of TILE_WCHUNK;
//   * heads[]  : one bit per edge, set where a local row starts (uint16 per 16 edges);
//   * tiles    : every block's rows are cut into row-aligned tiles of about equal estimated
//                cost (about three waves of CTAs over the device), one CTA each, launched
//                largest first so that the last wave holds the smallest tiles; every tile of a
//                block loads the same block values;
//   * wtab[]   : per tile, 33 (edge, row) pairs: warp w of the CTA owns the row-aligned edge
//                range [wtab[w].x, wtab[w+1].x) whose first row is wtab[w].y (equal estimated
//                cost per warp).
// The estimated cost of a row of L edges is 3 per edge, 1 per edge inside the chunks in which
// no row starts (the walk's fast path, about L - 512 edges once L >= 1024), and 2 for the row.
// A warp streams its range in chunks of TILE_WCHUNK edges, 16 consecutive edges per lane
// (two 16-byte loads), sums the source values of each lane's row pieces, and joins pieces of
// rows that cross lanes or chunks with a warp segmented scan.  Finished row sums go to a
// per-warp shared-memory stage and leave as coalesced stores to partial[row] in the
// partition's row numbering; the merge kernel (Fig. 5) reduces them.
#include <algorithm>
#include <vector>

#include "tc_common_dev.cuh"

namespace tc {

constexpr int WCH = TILE_WCHUNK;             // edges per warp chunk (16 per lane)
constexpr int TWARPS = TILE_THREADS / 32;

__host__ __device__ static inline size_t slice_bytes(int32_t W) { return ((size_t)W * 4 + 127) / 128 * 128; }

// per warp: WCH rows of stage plus 4 floats, so that the stage can be shifted to the alignment
// of the global rows it holds (bulk stores need matching 16-byte alignment on both sides)
constexpr int WSTAGE = WCH + 4;

size_t tile_smem_bytes(int32_t W) { return slice_bytes(W) + (size_t)TWARPS * WSTAGE * 4; }

int32_t tile_max_width(int max_smem_optin) {
    const int64_t budget = (int64_t)max_smem_optin - 1024 - (int64_t)TWARPS * WSTAGE * 4;
    int64_t W = budget / 4;
    W = W / 32 * 32;
    if (W > 65536) W = 65536;
    return W > 0 ? (int32_t)W : 0;
}

// The mbarrier and bulk-copy helpers (mbar_*, bulk_*) live in tc_common_dev.cuh.

struct TileArgs {
    const uint16_t *col16;
    const uint16_t *heads;
    const int32_t *tile_blk; // [ntiles]: block of every tile (in launch order)
    const int2 *wtab;        // [ntiles][TWARPS + 1]
    const float *contrib;
    int32_t V, W;
    float *partial;
    int *err;
};

// Loads lane `lane`'s 16 staged edges of the chunk at q0 (sources and row-start bits).
__device__ __forceinline__ void load_chunk(const TileArgs &t, int32_t q0, int lane, uint4 &c0, uint4 &c1, uint32_t &h) {
    const int32_t q = q0 + 16 * lane;
    const uint4 *p = reinterpret_cast<const uint4 *>(t.col16 + q);
    c0 = __ldg(p);
    c1 = __ldg(p + 1);
    h = __ldg(t.heads + (q >> 4));
}

// One warp's row-aligned range: edges [es, ee) of the staged stream, whose first row rs starts
// at es (Alg. 4 on the block values in `slice`); every row of it goes to partial[].
// Software pipeline: every chunk's loads are issued before the previous one is summed.
__device__ __forceinline__ void warp_walk(const TileArgs &t, const float *slice, float *stage_base, int32_t es,
                                          int32_t ee, int32_t rs, int lane) {
    int32_t rowbase = rs;                 // row started by the next head
    float carry = 0.0f;                   // value of the open row (rowbase - 1)
    bool open = false;                    // whether row rowbase-1 belongs to this warp
    const int32_t q_begin = es & ~(WCH - 1);
    uint4 nc0, nc1;
    uint32_t nh;
    load_chunk(t, q_begin, lane, nc0, nc1, nh);
    // Chunks in which no row starts (inside a row longer than a chunk, as hub destinations have)
    // only add to the open row: each lane keeps its share in racc, and the shares join the
    // carry (a fixed-order warp sum) before the next chunk that has a head.
    float racc = 0.0f;
    bool pend = false;  // warp-uniform: racc holds shares not yet in the carry
    for (int32_t q0 = q_begin; q0 < ee; q0 += WCH) {
        const uint4 c0 = nc0, c1 = nc1;
        uint32_t hd = nh;
        if (q0 + WCH < ee) load_chunk(t, q0 + WCH, lane, nc0, nc1, nh);
        const uint32_t words[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        const bool full = q0 >= es && q0 + WCH <= ee;  // whole chunk inside the warp's range (warp-uniform)
        if (full && __ballot_sync(0xffffffffu, hd != 0u) == 0u) {
            float s4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < 16; ++i) s4[i & 3] += slice[(words[i >> 1] >> (16 * (i & 1))) & 0xFFFFu];
            racc += (s4[0] + s4[1]) + (s4[2] + s4[3]);
            pend = true;
            continue;
        }
        if (pend) {
            float x = racc;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
            carry += x;
            racc = 0.0f;
            pend = false;
        }
        float val[16];
        if (full) {
#pragma unroll
            for (int i = 0; i < 16; ++i) val[i] = slice[(words[i >> 1] >> (16 * (i & 1))) & 0xFFFFu];
        } else {
            // valid edges of this lane: [max(es, e0), min(ee, e0 + 16))
            const int32_t e0 = q0 + 16 * lane;
            const int32_t lo_i = es - e0, hi_i = ee - e0;
            uint32_t valid = 0xFFFFu;
            if (lo_i > 0) valid = lo_i >= 16 ? 0u : (valid & (0xFFFFu << lo_i));
            if (hi_i < 16) valid = hi_i <= 0 ? 0u : (valid & ((1u << hi_i) - 1u));
            hd &= valid;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint32_t col = (words[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                val[i] = ((valid >> i) & 1u) ? slice[col] : 0.0f;
            }
        }
        // rows of this chunk: exclusive scan of head counts over lanes, from bit-sliced ballots
        // of the counts (at most 16, so five slices) instead of shuffles
        const int nh_l = __popc(hd);
        const uint32_t lt_mask = (1u << lane) - 1u;
        int before = 0, total = 0;  // heads in earlier lanes; heads in the chunk
#pragma unroll
        for (int bit = 0; bit < 5; ++bit) {
            const uint32_t m = __ballot_sync(0xffffffffu, (nh_l >> bit) & 1);
            before += __popc(m & lt_mask) << bit;
            total += __popc(m) << bit;
        }
        // walk the lane's 16 edges (branch-free): the piece before the first head goes to the
        // carry scan; every later head closes a whole row, written to the stage
        // stage[i] holds row rowbase - 1 + i; it starts (rowbase - 1) mod 4 floats into the
        // warp's buffer so that stage and partial[] agree modulo 16 bytes.  The previous
        // chunk's bulk store must have finished reading the buffer before it is rewritten.
        float *stage = stage_base + ((rowbase - 1) & 3);
        if (lane == 0) bulk_store_wait_read();
        __syncwarp();
        float seg = 0.0f, first = 0.0f;
        float *out = stage + before + 1;
        const uint32_t close_m = hd & (hd - 1u);  // heads after the lane's first: each closes a row
        const uint32_t first_m = hd & (0u - hd);  // the lane's first head
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            if ((close_m >> i) & 1u) *out++ = seg;  // close the row before this head
            if ((first_m >> i) & 1u) first = seg;   // the piece before the first head
            seg = ((hd >> i) & 1u) ? val[i] : seg + val[i];
        }
        const bool seen = hd != 0u;
        if (!seen) first = seg;
        // carry of the open row across lanes: segmented inclusive scan (Hillis-Steele). The
        // flag of lane l after the step of distance d is "a head in lanes (l - 2d, l]", read
        // from one ballot of the heads instead of being shuffled along with the values.
        const uint32_t F = __ballot_sync(0xffffffffu, seen);
        float v = seg;  // the open row's value at the lane's end (== first when no head)
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const float vp = __shfl_up_sync(0xffffffffu, v, d);
            const int lo = lane - d + 1;  // flag window of this lane before the step: [lo, lane]
            const uint32_t win = lo > 0 ? (F >> lo) & ((1u << d) - 1u) : F & ((2u << lane) - 1u);
            if (lane >= d && win == 0u) v += vp;
        }
        const bool f = (F & ((2u << lane) - 1u)) != 0u;  // a head in lanes [0, lane]
        // open-row value at the end of lane l: f ? v : carry + v (no head yet: the chunk's
        // carry flows through); the row closed at lane l's first head gets X(l-1) + first
        const float vprev = __shfl_up_sync(0xffffffffu, v, 1);
        const bool fprev = (F & lt_mask) != 0u;
        const float xprev = (lane == 0) ? carry : (fprev ? vprev : carry + vprev);
        if (seen) stage[before] = xprev + first;
        const float xlast = __shfl_sync(0xffffffffu, f ? v : carry + v, 31);
        // Rows rowbase - 1 + [i0, total) leave: stage[0] is the open row only when it belongs
        // to this warp.  The 16-byte aligned middle goes out as one bulk store (TMA) issued by
        // lane 0 after every lane's proxy fence; the at most 3 + 3 rows at the ends are plain
        // stores.
        fence_proxy_async_smem();
        __syncwarp();
        {
            const int32_t r0 = rowbase - 1;
            const int32_t g0 = r0 + (open ? 0 : 1), g1 = r0 + total;
            const int32_t ga = (g0 + 3) & ~3, gb = g1 & ~3;
            if (g1 < ga) {  // no aligned group of 4 inside
                if (g0 + lane < g1) t.partial[g0 + lane] = stage[g0 + lane - r0];
            } else {
                if (g0 + lane < ga) t.partial[g0 + lane] = stage[g0 + lane - r0];
                if (gb + lane < g1) t.partial[gb + lane] = stage[gb + lane - r0];
                if (gb > ga && lane == 0) bulk_store_s2g(t.partial + ga, stage + (ga - r0), (uint32_t)(gb - ga) * 4u);
            }
        }
        if (total > 0) open = true;
        rowbase += total;
        carry = xlast;
    }
    if (pend) {
        float x = racc;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
        carry += x;
    }
    if (open && lane == 0) t.partial[rowbase - 1] = carry;
}

__global__ void __launch_bounds__(TILE_THREADS, 1) k_tile_gather(TileArgs t) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t slice_bar;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t tile = blockIdx.x;
    const int32_t b = t.tile_blk[tile];
    float *slice = reinterpret_cast<float *>(smem);
    float *stage_base = reinterpret_cast<float *>(smem + slice_bytes(t.W)) + warp * WSTAGE;
    // ---- the block's contributions -> shared memory (bulk copies on one mbarrier) ----
    if (tid == 0) {
        mbar_init(&slice_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // launched programmatically after the merge: the contributions are its output.  No early
    // trigger here: the merge's CTAs then launch as the tiles finish and do not sit on SMs the
    // last wave of tiles could use (measured: 0.6% per step against triggering at the start).
    pdl_wait();
    __syncthreads();
    if (tid == 0) {
        const int64_t lo = (int64_t)b * t.W;
        const int64_t n = ((int64_t)t.V - lo) < t.W ? ((int64_t)t.V - lo) : t.W;
        const uint32_t bytes = (uint32_t)((n * 4 + 15) & ~15LL);
        mbar_expect_tx(&slice_bar, bytes);
        for (uint32_t off = 0; off < bytes; off += 16384) {
            const uint32_t part = (bytes - off) < 16384u ? (bytes - off) : 16384u;
            bulk_g2s(reinterpret_cast<unsigned char *>(slice) + off,
                     reinterpret_cast<const unsigned char *>(t.contrib + lo) + off, part, &slice_bar);
        }
    }
    // every thread waits for the copy (bounded); on a timeout the flag is set and all leave
    if (!mbar_wait(&slice_bar, 0, t.err, 1)) return;
    const int2 w0 = t.wtab[(int64_t)tile * (TWARPS + 1) + warp];
    const int2 w1 = t.wtab[(int64_t)tile * (TWARPS + 1) + warp + 1];
    if (w0.x < w1.x) warp_walk(t, slice, stage_base, w0.x, w1.x, w0.y, lane);
    if (lane == 0) bulk_store_wait_all();  // the stage must outlive the bulk stores reading it
}

// ---------------------------------------------------------------------------------------------
// building the staged format from a base partition
// ---------------------------------------------------------------------------------------------
// Block b's edges are contiguous in the partition and keep their order in the staged stream, so
// filling it is a straight copy over all edges: edge i of block b = colidx[i] / W goes to
// col16[i + delta[b]] = colidx[i] - b W, with delta[b] = pbase[b] - blk_edges[b].  Edge-parallel
// over the whole stream, so one block holding most of the edges gets the whole grid.
__global__ void k_tile_copy(const int32_t *colidx, int64_t E, DivBy W, int32_t Wi, const int64_t *delta,
                            uint16_t *col16) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    // eight independent loads in flight per thread, then their stores
    for (; i + 7 * stride < E; i += 8 * stride) {
        int32_t c[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = __ldg(colidx + i + k * stride);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int32_t b = div_apply(c[k], W);
            col16[i + k * stride + __ldg(delta + b)] = (uint16_t)(c[k] - b * Wi);
        }
    }
    for (; i < E; i += stride) {
        const int32_t c = __ldg(colidx + i), b = div_apply(c, W);
        col16[i + __ldg(delta + b)] = (uint16_t)(c - b * Wi);
    }
}

// A head bit at the first staged edge of every local row (row r's block is that of its first
// edge's column).  A warp's 32 rows are consecutive, so their head positions increase with the
// lane: lanes whose heads share a 32-bit word OR their bits together (segmented shuffle
// reduction) and one atomic per word remains.
__global__ void k_tile_heads(const int32_t *rowptr, const int32_t *colidx, int64_t R, DivBy W, const int64_t *delta,
                             uint32_t *heads32) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // four groups of 32 rows per step: their row offsets are loaded together
    for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); r0 < R; r0 += 4 * stride) {
        int32_t s4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t r = r0 + k * stride + lane;
            s4[k] = r < R ? rowptr[r] : 0;
        }
        int64_t d4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t r = r0 + k * stride + lane;
            d4[k] = r < R ? (int64_t)s4[k] + __ldg(delta + div_apply(__ldg(colidx + s4[k]), W)) : -1;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t word = 0xFFFFFFFFu, bit = 0u;  // lanes past the rows: a group of their own, no atomic
            if (d4[k] >= 0) {
                word = (uint32_t)(d4[k] >> 5);
                bit = 1u << (d4[k] & 31);
            }
            uint32_t v = bit;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_down_sync(0xffffffffu, v, d);
                const uint32_t wy = __shfl_down_sync(0xffffffffu, word, d);
                if (lane + d < 32 && wy == word) v |= y;
            }
            const uint32_t wprev = __shfl_up_sync(0xffffffffu, word, 1);
            if (bit && (lane == 0 || wprev != word)) atomicOr(heads32 + word, v);
        }
    }
}

// Estimated cost of every local row (see the top of the file); w[R] = 0 closes the scan.
__global__ void k_row_weights(const int32_t *rowptr, int64_t R, int32_t *w) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x) {
        if (r == R) {
            w[R] = 0;
            continue;
        }
        const int32_t L = rowptr[r + 1] - rowptr[r];
        const int32_t fast = L >= 1024 ? ((L >> 9) - 1) << 9 : 0;
        w[r] = 3 * L - 2 * fast + 2;
    }
}

// First row r in [lo, hi] with cum[r] >= target (cum ascending; cum[hi] >= target).
__device__ __forceinline__ int64_t first_row_at(const int64_t *cum, int64_t lo, int64_t hi, int64_t target) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cum[mid] < target) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Weight prefix at every block's first row: cw[b] = cum[blk_rows[b]], b in [0, B].
__global__ void k_block_weights(const int64_t *cum, const int64_t *blk_rows, int32_t B, int64_t *cw) {
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += gridDim.x * blockDim.x) cw[b] = cum[blk_rows[b]];
}

// Rows and cost of every tile: tile k of the n tiles of block b spans the rows whose weight prefix
// lies in the k-th n-th of the block's weight range (row-aligned, rounded up).
__global__ void k_tile_rows(const int64_t *cum, const int64_t *blk_rows, const int4 *tiles, int32_t ntiles,
                            int2 *rows, int64_t *cost) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
        const int4 tt = tiles[t];  // (block, k, n, 0)
        const int64_t br0 = blk_rows[tt.x], br1 = blk_rows[tt.x + 1];
        const int64_t c0 = cum[br0], c1 = cum[br1];
        const int64_t r0 = first_row_at(cum, br0, br1, c0 + ((c1 - c0) * tt.y + tt.z - 1) / tt.z);
        const int64_t r1 = first_row_at(cum, br0, br1, c0 + ((c1 - c0) * (tt.y + 1) + tt.z - 1) / tt.z);
        rows[t] = make_int2((int32_t)r0, (int32_t)r1);
        cost[t] = cum[r1] - cum[r0];
    }
}

// Warp ranges of every tile (rows [r0, r1) of block b): warp w starts at the first row whose
// weight prefix reaches cum[r0] + (cum[r1] - cum[r0]) w / TWARPS (rounded up); stored as
// (position in the staged stream, row).
__global__ void k_tile_wtab(const int32_t *rowptr, const int64_t *cum, const int64_t *blk_edges, const int64_t *pbase,
                            const int32_t *tile_blk, const int2 *tile_rows, int32_t ntiles, int2 *wtab) {
    const int64_t total = (int64_t)ntiles * (TWARPS + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t tile = (int32_t)(t / (TWARPS + 1)), w = (int32_t)(t % (TWARPS + 1));
        const int32_t b = tile_blk[tile];
        const int64_t r0 = tile_rows[tile].x, r1 = tile_rows[tile].y;
        const int64_t c0 = cum[r0], c1 = cum[r1];
        const int64_t r = first_row_at(cum, r0, r1, c0 + ((c1 - c0) * w + TWARPS - 1) / TWARPS);
        const int64_t edge = rowptr[r];
        wtab[t] = make_int2((int32_t)(pbase[b] + (edge - blk_edges[b])), (int32_t)r);
    }
}

int build_tiles(tc_part *p, int sms, cudaStream_t s) {
    p->tiled = false;
    const int64_t R = p->R;
    const int32_t B = p->B;
    if (R == 0 || p->E == 0) return TC_OK;
    int64_t *h_pbase = new (std::nothrow) int64_t[B + 1];
    if (!h_pbase) return fail(TC_ERR_OOM, "host allocation failed");
    h_pbase[0] = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t ne = p->h_blk_edges[b + 1] - p->h_blk_edges[b];
        h_pbase[b + 1] = h_pbase[b] + (ne + WCH - 1) / WCH * WCH;
    }
    const int64_t npad = h_pbase[B];
    if (npad >= INT32_MAX - WCH) {
        delete[] h_pbase;
        return TC_OK;  // padded stream beyond int32 positions: keep the unstaged gather
    }
    DevBuf pbase, blk_edges;
    int st = pbase.alloc((size_t)(B + 1) * 8);
    if (st == TC_OK) st = blk_edges.alloc((size_t)(B + 1) * 8);
    cudaError_t e = cudaSuccess;
    if (st == TC_OK) e = cudaMemcpyAsync(pbase.p, h_pbase, (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, s);
    if (st == TC_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(blk_edges.p, p->h_blk_edges, (size_t)(B + 1) * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] h_pbase;
    if (st != TC_OK) return st;
    if (e != cudaSuccess) return fail(TC_ERR_CUDA, "build_tiles: %s", cudaGetErrorString(e));
    // + one chunk of slack: the software pipeline never reads past npad, but keep loads in bounds
    TC_TRY(p->col16.alloc((size_t)(npad + WCH) * 2));
    TC_TRY(p->heads.alloc((size_t)(npad + WCH) / 8 + 64));
    TC_CUDA(cudaMemsetAsync(p->col16.p, 0, (size_t)(npad + WCH) * 2, s));
    TC_CUDA(cudaMemsetAsync(p->heads.p, 0, (size_t)(npad + WCH) / 8 + 64, s));
    // tiles: the rows of every block with edges are cut into n_b = max(1, round(cost_b / T)) tiles
    // of equal estimated cost, T = the total over three waves of one CTA per SM
    DevBuf wrow, cum, cw;
    TC_TRY(wrow.alloc(((size_t)R + 1) * 4));
    TC_TRY(cum.alloc(((size_t)R + 1) * 8));
    TC_TRY(cw.alloc(((size_t)B + 1) * 8));
    k_row_weights<<<sms * 8, 256, 0, s>>>(p->rowptr.as<int32_t>(), R, wrow.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32_to_i64(wrow.as<int32_t>(), R + 1, cum.as<int64_t>(), s));
    wrow.release();
    k_block_weights<<<(B + 256) / 256, 256, 0, s>>>(cum.as<int64_t>(), p->blk_rows_dev.as<int64_t>(), B,
                                                    cw.as<int64_t>());
    TC_LAUNCH_CHECK();
    std::vector<int64_t> h_cw((size_t)B + 1);
    TC_CUDA(cudaMemcpyAsync(h_cw.data(), cw.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    const int64_t T = h_cw[B] / (3LL * sms) > 0 ? h_cw[B] / (3LL * sms) : 1;
    std::vector<int4> h_tiles;
    for (int32_t b = 0; b < B; ++b) {
        if (p->h_blk_edges[b + 1] == p->h_blk_edges[b]) continue;
        int64_t n = (h_cw[b + 1] - h_cw[b] + T / 2) / T;
        if (n < 1) n = 1;
        if (n > p->h_blk_rows[b + 1] - p->h_blk_rows[b]) n = p->h_blk_rows[b + 1] - p->h_blk_rows[b];
        for (int64_t k = 0; k < n; ++k) h_tiles.push_back(make_int4(b, (int)k, (int)n, 0));
    }
    const int64_t ntiles = (int64_t)h_tiles.size();
    if (ntiles * (TWARPS + 1) > INT32_MAX) return fail(TC_ERR_UNSUPPORTED, "build_tiles: too many tiles");
    DevBuf tiles_dev, rows0, cost, rows_lpt;
    const size_t nt = (size_t)(ntiles > 0 ? ntiles : 1);
    TC_TRY(tiles_dev.alloc(nt * 16));
    TC_TRY(rows0.alloc(nt * 8));
    TC_TRY(rows_lpt.alloc(nt * 8));
    TC_TRY(cost.alloc(nt * 8));
    TC_TRY(p->tile_blk.alloc(nt * 4));
    if (ntiles > 0) {
        TC_CUDA(cudaMemcpyAsync(tiles_dev.p, h_tiles.data(), (size_t)ntiles * 16, cudaMemcpyHostToDevice, s));
        k_tile_rows<<<(unsigned)((ntiles + 255) / 256), 256, 0, s>>>(cum.as<int64_t>(), p->blk_rows_dev.as<int64_t>(),
                                                                     tiles_dev.as<int4>(), (int32_t)ntiles,
                                                                     rows0.as<int2>(), cost.as<int64_t>());
        TC_LAUNCH_CHECK();
        // launch order: largest estimated cost first (ties by position), so that the CTAs of the
        // last wave run the smallest tiles
        std::vector<int64_t> h_cost((size_t)ntiles);
        std::vector<int2> h_rows((size_t)ntiles);
        TC_CUDA(cudaMemcpyAsync(h_cost.data(), cost.p, (size_t)ntiles * 8, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaMemcpyAsync(h_rows.data(), rows0.p, (size_t)ntiles * 8, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> order((size_t)ntiles);
        for (int64_t i = 0; i < ntiles; ++i) order[(size_t)i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t c) { return h_cost[(size_t)a] > h_cost[(size_t)c]; });
        std::vector<int32_t> h_blk((size_t)ntiles);
        std::vector<int2> h_rows_lpt((size_t)ntiles);
        for (int64_t i = 0; i < ntiles; ++i) {
            h_blk[(size_t)i] = h_tiles[(size_t)order[(size_t)i]].x;
            h_rows_lpt[(size_t)i] = h_rows[(size_t)order[(size_t)i]];
        }
        TC_CUDA(cudaMemcpyAsync(p->tile_blk.p, h_blk.data(), (size_t)ntiles * 4, cudaMemcpyHostToDevice, s));
        TC_CUDA(cudaMemcpyAsync(rows_lpt.p, h_rows_lpt.data(), (size_t)ntiles * 8, cudaMemcpyHostToDevice, s));
        TC_TRY(p->wtab.alloc(nt * (TWARPS + 1) * 8));
        k_tile_wtab<<<(unsigned)((ntiles * (TWARPS + 1) + 255) / 256), 256, 0, s>>>(
            p->rowptr.as<int32_t>(), cum.as<int64_t>(), blk_edges.as<int64_t>(), pbase.as<int64_t>(),
            p->tile_blk.as<int32_t>(), rows_lpt.as<int2>(), (int32_t)ntiles, p->wtab.as<int2>());
        TC_LAUNCH_CHECK();
        TC_CUDA(cudaStreamSynchronize(s));  // the host vectors above must outlive their copies
    }
    p->ntiles = (int32_t)ntiles;
    // the staged stream and its row-head bits, edge- and row-parallel over the whole partition
    std::vector<int64_t> h_delta((size_t)B);
    {
        int64_t pb = 0;
        for (int32_t b = 0; b < B; ++b) {
            h_delta[(size_t)b] = pb - p->h_blk_edges[b];
            pb += (p->h_blk_edges[b + 1] - p->h_blk_edges[b] + WCH - 1) / WCH * WCH;
        }
    }
    DevBuf delta;
    TC_TRY(delta.alloc((size_t)B * 8));
    TC_CUDA(cudaMemcpyAsync(delta.p, h_delta.data(), (size_t)B * 8, cudaMemcpyHostToDevice, s));
    k_tile_copy<<<sms * 8, 256, 0, s>>>(p->colidx.as<int32_t>(), p->E, div_by(p->W), p->W, delta.as<int64_t>(),
                                        p->col16.as<uint16_t>());
    TC_LAUNCH_CHECK();
    k_tile_heads<<<sms * 8, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->colidx.as<int32_t>(), R, div_by(p->W),
                                         delta.as<int64_t>(), p->heads.as<uint32_t>());
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaStreamSynchronize(s));
    p->padded_edges = npad;
    p->tiled = true;
    return TC_OK;
}

int launch_tiled_gather(const tc_part *p, const float *contrib, int *err_flag, cudaStream_t s, int *launches) {
    const size_t smem = tile_smem_bytes(p->W);
    TC_CUDA(cudaFuncSetAttribute(k_tile_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (p->ntiles == 0) return TC_OK;  // no edges: no partial sums exist
    TileArgs t;
    t.col16 = p->col16.as<uint16_t>();
    t.heads = p->heads.as<uint16_t>();
    t.tile_blk = p->tile_blk.as<int32_t>();
    t.wtab = p->wtab.as<int2>();
    t.contrib = contrib;
    t.V = p->V;
    t.W = p->W;
    t.partial = const_cast<float *>(p->partial.as<float>());
    t.err = err_flag;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p->ntiles);
    cfg.blockDim = dim3(TILE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    TC_CUDA(cudaLaunchKernelEx(&cfg, k_tile_gather, t));
    ++*launches;
    return TC_OK;
}

}  // namespace tc
