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
//   * items    : every block's staged edges are cut into items of ITEM_EDGES (whole warp
//                chunks; the last item of a block may be shorter); one persistent CTA per SM
//                holds one block's values at a time and its warps draw that block's items from
//                the block's work counter; a CTA starts in its own stretch of blocks (in
//                proportion to their edges) and moves on to the next block with items left once
//                its block runs dry, so no CTA idles while work remains and few blocks are
//                loaded twice;
//   * a row may cross items: an item records the piece of the row open at its start (head)
//     and the row open at its end with its piece (tail), and a fix-up pass adds every tail to
//     the heads of the items that follow it, in item order (deterministic).
// A warp streams its range in chunks of TILE_WCHUNK edges, 16 consecutive edges per lane
// (two 16-byte loads), sums the source values of each lane's row pieces, and joins pieces of
// rows that cross lanes or chunks with a warp segmented scan.  Finished row sums go to a
// per-warp shared-memory stage and leave as coalesced stores to partial[row] in the
// partition's row numbering; the merge kernel (Fig. 5) reduces them.
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
    const int4 *items;       // [nitems]: (first staged edge, end, first row, 0), block after block
    const int32_t *ibase;    // [B + 1]: first item of every block
    const int32_t *cta_blk;  // [gridDim.x]: the block every CTA starts in
    int32_t B;
    unsigned *bq;            // [B + 1]: items handed out per block; bq[B] counts finished CTAs
    float *headval;          // [nitems]: the item's piece of the row open at its start
    float *tailval;          // [nitems]: the item's piece of the row open at its end
    int32_t *tailrow;        // [nitems]: that row, or -1 when no row starts in the item
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

// One warp's item: edges [es, ee) of the staged stream (es at a chunk start), the first row
// starting in it rs (Alg. 4 on the block values in `slice`).  Rows that start and end inside
// the item go to partial[]; the pieces of the rows open at its two ends go to the item's records.
// Software pipeline: (nc0, nc1, nh) hold the item's first chunk on entry; every chunk's loads
// are issued before the previous one is summed, and the last chunk's loads fetch the first chunk
// of the warp's next item (at next_es, if >= 0), which (nc0, nc1, nh) then hold on return.
__device__ __forceinline__ void warp_walk(const TileArgs &t, const float *slice, float *stage_base, int32_t es,
                                          int32_t ee, int32_t rs, int lane, int32_t item, uint4 &nc0, uint4 &nc1,
                                          uint32_t &nh, int32_t next_es) {
    int32_t rowbase = rs;                 // row started by the next head
    float carry = 0.0f;                   // value of the open row (rowbase - 1)
    bool open = false;                    // whether row rowbase-1 belongs to this warp
    const int32_t q_begin = es & ~(WCH - 1);
    // Chunks in which no row starts (inside a row longer than a chunk, as hub destinations have)
    // only add to the open row: each lane keeps its share in racc, and the shares join the
    // carry (a fixed-order warp sum) before the next chunk that has a head.
    float racc = 0.0f;
    bool pend = false;  // warp-uniform: racc holds shares not yet in the carry
    for (int32_t q0 = q_begin; q0 < ee; q0 += WCH) {
        const uint4 c0 = nc0, c1 = nc1;
        uint32_t hd = nh;
        if (q0 + WCH < ee) load_chunk(t, q0 + WCH, lane, nc0, nc1, nh);
        else if (next_es >= 0) load_chunk(t, next_es, lane, nc0, nc1, nh);
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
        if (!open && total > 0 && lane == 0) t.headval[item] = stage[0];  // the row open at es
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
    if (lane == 0) {
        if (open) {  // the last row started here runs to the end of the item (or beyond)
            t.tailval[item] = carry;
            t.tailrow[item] = rowbase - 1;
        } else {     // no row starts in the item: all of it continues the row open at es
            t.headval[item] = carry;
            t.tailrow[item] = -1;
        }
    }
}

// partial[tailrow[i]] = tailval[i] + the heads of the items that follow i up to and including the
// first one in which a row starts (a block's first item starts with a row, so a row never takes
// a head from another block).
__global__ void k_item_fixup(const float *headval, const float *tailval, const int32_t *tailrow, int32_t nitems,
                             float *partial) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nitems; i += gridDim.x * blockDim.x) {
        const int32_t r = tailrow[i];
        if (r < 0) continue;
        float v = tailval[i];
        int32_t j = i + 1;
        while (j < nitems && tailrow[j] < 0) v += headval[j++];
        if (j < nitems) v += headval[j];
        partial[r] = v;
    }
}

__global__ void __launch_bounds__(TILE_THREADS, 1) k_tile_gather(TileArgs t) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t slice_bar;
    __shared__ int32_t s_b;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *slice = reinterpret_cast<float *>(smem);
    float *stage_base = reinterpret_cast<float *>(smem + slice_bytes(t.W)) + warp * WSTAGE;
    if (tid == 0) {
        mbar_init(&slice_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    int32_t b = t.cta_blk[blockIdx.x];
    for (;;) {
        // the first block from b on that still has items to hand out
        if (tid == 0) {
            while (b < t.B && *(volatile unsigned *)(t.bq + b) >= (unsigned)(t.ibase[b + 1] - t.ibase[b])) ++b;
            s_b = b;
        }
        __syncthreads();  // also: every warp is done with the previous block's values
        b = s_b;
        if (b >= t.B) break;
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
        // every thread waits for the copy (bounded); if any thread gives up, the flag is set and
        // the whole CTA leaves together
        const bool ok = mbar_wait(&slice_bar, phase, t.err, 1);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) break;
        // Each warp draws the block's items one at a time.  The next item's index is drawn while
        // the current one is summed, and its descriptor and first chunk load during the current
        // item's last chunk, so no draw or load waits between items.
        const int32_t i0 = t.ibase[b], ni = t.ibase[b + 1] - i0;
        int32_t cur = 0;
        if (lane == 0) cur = (int32_t)atomicAdd(t.bq + b, 1u);
        cur = __shfl_sync(0xffffffffu, cur, 0);
        if (cur < ni) {
            int4 dc = t.items[i0 + cur];
            uint4 nc0, nc1;
            uint32_t nh;
            load_chunk(t, dc.x, lane, nc0, nc1, nh);
            int32_t drawn = 0;
            if (lane == 0) drawn = (int32_t)atomicAdd(t.bq + b, 1u);
            for (;;) {
                const int32_t nxt = __shfl_sync(0xffffffffu, drawn, 0);
                int4 dn = make_int4(-1, -1, 0, 0);
                if (nxt < ni) {
                    dn = t.items[i0 + nxt];
                    if (lane == 0) drawn = (int32_t)atomicAdd(t.bq + b, 1u);
                }
                warp_walk(t, slice, stage_base, dc.x, dc.y, dc.z, lane, i0 + cur, nc0, nc1, nh, dn.x);
                if (nxt >= ni) break;
                cur = nxt;
                dc = dn;
            }
        }
        ++b;
    }
    if (lane == 0) bulk_store_wait_all();  // the stage must outlive the bulk stores reading it
    // the last CTA to finish re-arms the counters (every CTA has drawn its last item by now)
    __syncthreads();
    __shared__ bool last;
    if (tid == 0) {
        __threadfence();
        last = atomicAdd(t.bq + t.B, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last)
        for (int32_t k = tid; k <= t.B; k += TILE_THREADS) t.bq[k] = 0u;
}

// ---------------------------------------------------------------------------------------------
// building the staged format from a base partition
// ---------------------------------------------------------------------------------------------
// Block b's edges are contiguous in the partition and keep their order in the staged stream, so
// filling it is a straight copy: col16[pbase[b] + (i - eb)] = colidx[i] - b*W (grid.y strides
// over blocks, grid.x over a block's edges).
__global__ void k_tile_copy(const int32_t *colidx, const int64_t *blk_edges, const int64_t *pbase, int32_t B,
                            int32_t W, uint16_t *col16) {
    for (int32_t b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t eb = blk_edges[b], ee = blk_edges[b + 1];
        const int64_t off = pbase[b] - eb;
        const int32_t base = b * W;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        int64_t i = eb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        // eight independent loads in flight per thread, then their stores
        for (; i + 7 * stride < ee; i += 8 * stride) {
            int32_t c[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) c[k] = __ldg(colidx + i + k * stride);
#pragma unroll
            for (int k = 0; k < 8; ++k) col16[i + k * stride + off] = (uint16_t)(c[k] - base);
        }
        for (; i < ee; i += stride) col16[i + off] = (uint16_t)(__ldg(colidx + i) - base);
    }
}

// A head bit at the first staged edge of every local row.  A warp's 32 rows are consecutive, so
// their head positions increase with the lane: lanes whose heads share a 32-bit word OR their
// bits together (segmented shuffle reduction) and one atomic per word remains.
__global__ void k_tile_heads(const int32_t *rowptr, const int64_t *blk_rows, const int64_t *blk_edges,
                             const int64_t *pbase, int32_t B, uint32_t *heads32) {
    const int lane = threadIdx.x & 31;
    for (int32_t b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t r1 = blk_rows[b + 1];
        const int64_t off = pbase[b] - blk_edges[b];
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        // four groups of 32 rows per step: their row offsets are loaded together
        for (int64_t r0 = blk_rows[b] + blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); r0 < r1;
             r0 += 4 * stride) {
            int32_t s4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t r = r0 + k * stride + lane;
                s4[k] = r < r1 ? rowptr[r] : 0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t r = r0 + k * stride + lane;
                uint32_t word = 0xFFFFFFFFu, bit = 0u;  // lanes past the block: a group of their own, no atomic
                if (r < r1) {
                    const int64_t dst = s4[k] + off;
                    word = (uint32_t)(dst >> 5);
                    bit = 1u << (dst & 31);
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
}

// Items of every block: item k of block b holds the staged edges [pbase[b] + k ITEM_EDGES,
// min(that + ITEM_EDGES, pbase[b] + edges of b)); its first row is the first row of the block
// starting at or after that edge (blk_rows[b + 1] when none does).  Stored as (staged start,
// staged end, first row, 0).
__global__ void k_items(const int32_t *rowptr, const int64_t *blk_rows, const int64_t *blk_edges, const int64_t *pbase,
                        const int32_t *ibase, const int32_t *item_blk, int32_t nitems, int4 *items) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nitems; t += gridDim.x * blockDim.x) {
        const int32_t b = item_blk[t], k = t - ibase[b];
        const int64_t eb = blk_edges[b], ne = blk_edges[b + 1] - eb;
        const int64_t off = (int64_t)k * ITEM_EDGES;
        const int64_t end = off + ITEM_EDGES < ne ? off + ITEM_EDGES : ne;
        int64_t lo = blk_rows[b], hi = blk_rows[b + 1];  // rowptr[blk_rows[b + 1]] = blk_edges[b + 1]
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)rowptr[mid] < eb + off) lo = mid + 1; else hi = mid;
        }
        items[t] = make_int4((int32_t)(pbase[b] + off), (int32_t)(pbase[b] + end), (int32_t)lo, 0);
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
    // items: ceil(edges / ITEM_EDGES) per block; the CTAs' starting blocks split the edges evenly
    std::vector<int32_t> h_ibase((size_t)B + 1, 0), h_item_blk, h_cta_blk;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t ne = p->h_blk_edges[b + 1] - p->h_blk_edges[b];
        const int64_t n = (ne + ITEM_EDGES - 1) / ITEM_EDGES;
        if ((int64_t)h_ibase[b] + n > INT32_MAX / 2) return fail(TC_ERR_UNSUPPORTED, "build_tiles: too many items");
        h_ibase[b + 1] = h_ibase[b] + (int32_t)n;
        for (int64_t k = 0; k < n; ++k) h_item_blk.push_back(b);
    }
    const int32_t nitems = h_ibase[B];
    const int32_t G = (int32_t)(nitems < sms ? nitems : sms);
    for (int32_t c = 0, b = 0; c < G; ++c) {
        const int64_t at = p->E * c / G;  // CTA c starts in the block holding edge c E / G
        while (b + 1 < B && p->h_blk_edges[b + 1] <= at) ++b;
        h_cta_blk.push_back(b);
    }
    TC_TRY(p->items.alloc((size_t)(nitems > 0 ? nitems : 1) * 16));
    TC_TRY(p->ibase.alloc(((size_t)B + 1) * 4));
    TC_TRY(p->cta_blk.alloc((size_t)(G > 0 ? G : 1) * 4));
    TC_TRY(p->bq.alloc(((size_t)B + 1) * 4));
    TC_TRY(p->headval.alloc((size_t)(nitems > 0 ? nitems : 1) * 4));
    TC_TRY(p->tailval.alloc((size_t)(nitems > 0 ? nitems : 1) * 4));
    TC_TRY(p->tailrow.alloc((size_t)(nitems > 0 ? nitems : 1) * 4));
    TC_CUDA(cudaMemsetAsync(p->bq.p, 0, ((size_t)B + 1) * 4, s));
    DevBuf item_blk;
    TC_TRY(item_blk.alloc((size_t)(nitems > 0 ? nitems : 1) * 4));
    TC_CUDA(cudaMemcpyAsync(p->ibase.p, h_ibase.data(), ((size_t)B + 1) * 4, cudaMemcpyHostToDevice, s));
    if (nitems > 0)
        TC_CUDA(cudaMemcpyAsync(item_blk.p, h_item_blk.data(), (size_t)nitems * 4, cudaMemcpyHostToDevice, s));
    if (G > 0) TC_CUDA(cudaMemcpyAsync(p->cta_blk.p, h_cta_blk.data(), (size_t)G * 4, cudaMemcpyHostToDevice, s));
    p->nitems = nitems;
    p->gather_ctas = G;
    // grid.y over blocks, grid.x over each block's share: about 8 CTAs per SM in all
    const int gy = B < 65535 ? B : 65535;
    const dim3 grid((unsigned)((sms * 8 + gy - 1) / gy), (unsigned)gy);
    k_tile_copy<<<grid, 256, 0, s>>>(p->colidx.as<int32_t>(), blk_edges.as<int64_t>(), pbase.as<int64_t>(), B, p->W,
                                     p->col16.as<uint16_t>());
    TC_LAUNCH_CHECK();
    k_tile_heads<<<grid, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->blk_rows_dev.as<int64_t>(), blk_edges.as<int64_t>(),
                                      pbase.as<int64_t>(), B, p->heads.as<uint32_t>());
    TC_LAUNCH_CHECK();
    if (nitems > 0) {
        k_items<<<(nitems + 255) / 256, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->blk_rows_dev.as<int64_t>(),
                                                     blk_edges.as<int64_t>(), pbase.as<int64_t>(), p->ibase.as<int32_t>(),
                                                     item_blk.as<int32_t>(), nitems, p->items.as<int4>());
        TC_LAUNCH_CHECK();
    }
    TC_CUDA(cudaStreamSynchronize(s));
    p->padded_edges = npad;
    p->tiled = true;
    return TC_OK;
}

int launch_tiled_gather(const tc_part *p, const float *contrib, int *err_flag, cudaStream_t s, int *launches) {
    const size_t smem = tile_smem_bytes(p->W);
    TC_CUDA(cudaFuncSetAttribute(k_tile_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (p->nitems == 0) return TC_OK;  // no edges: every partial sum is empty (none exist)
    TileArgs t;
    t.col16 = p->col16.as<uint16_t>();
    t.heads = p->heads.as<uint16_t>();
    t.items = p->items.as<int4>();
    t.ibase = p->ibase.as<int32_t>();
    t.cta_blk = p->cta_blk.as<int32_t>();
    t.B = p->B;
    t.bq = const_cast<unsigned *>(p->bq.as<unsigned>());
    t.headval = const_cast<float *>(p->headval.as<float>());
    t.tailval = const_cast<float *>(p->tailval.as<float>());
    t.tailrow = const_cast<int32_t *>(p->tailrow.as<int32_t>());
    t.contrib = contrib;
    t.V = p->V;
    t.W = p->W;
    t.partial = const_cast<float *>(p->partial.as<float>());
    t.err = err_flag;
    k_tile_gather<<<p->gather_ctas, TILE_THREADS, smem, s>>>(t);
    TC_LAUNCH_CHECK();
    k_item_fixup<<<(p->nitems + 255) / 256 < 4 * p->gather_ctas ? (p->nitems + 255) / 256 : 4 * p->gather_ctas, 256, 0,
                   s>>>(t.headval, t.tailval, t.tailrow, p->nitems, t.partial);
    TC_LAUNCH_CHECK();
    *launches += 2;
    return TC_OK;
}

}  // namespace tc
