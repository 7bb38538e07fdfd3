// Shared-memory staged TOCAB gather (Alg. 4 with the block's vertex values on chip).
//
// The paper sizes a block so that its contributions fit in the last-level cache (Sec. 3.1).
// On GB300 the whole contribution vector of a scale-24 graph already fits in the 135 MB L2,
// and the random requests themselves become the bound (one L1/L2 sector request per edge).
// This format sizes a block so that its contributions fit in one CTA's shared memory instead,
// where a random warp gather costs a few bank cycles:
//   * one CTA per block; the block's contributions are copied into shared memory with bulk
//     asynchronous copies (TMA, cp.async.bulk) completing on an mbarrier;
//   * col16[]  : uint16 source offset inside the block (source - b*W), each block's edges
//                padded to a multiple of TILE_WCHUNK;
//   * heads[]  : one bit per edge, set where a local row starts (uint16 per 16 edges);
//   * wtab[]   : per block, 33 (edge, row) pairs: warp w of the CTA owns the row-aligned edge
//                range [wtab[w].x, wtab[w+1].x) whose first row is wtab[w].y.
// A warp streams its range in chunks of TILE_WCHUNK edges, 16 consecutive edges per lane
// (two 16-byte loads), sums the source values of each lane's row pieces, and joins pieces of
// rows that cross lanes or chunks with a warp segmented scan.  Finished row sums go to a
// per-warp shared-memory stage and leave as coalesced stores to partial[row] in the
// partition's row numbering; the merge kernel (Fig. 5) reduces them.
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

// ---- PTX helpers: mbarrier and bulk asynchronous copies -------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~2^31 cycles (about a second), records `code` in *err.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > (1LL << 31)) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bulk store shared -> global (TMA unit), one per call, committed as its own group; both
// addresses 16-byte aligned and the size a multiple of 16.
__device__ __forceinline__ void bulk_store_s2g(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_addr(ssrc)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until this thread's bulk stores have read their shared-memory sources.
__device__ __forceinline__ void bulk_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Waits until this thread's bulk stores are complete.
__device__ __forceinline__ void bulk_store_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's generic-proxy shared-memory writes before later bulk-copy reads.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct TileArgs {
    const uint16_t *col16;
    const uint16_t *heads;
    const int2 *wtab;      // [B][TWARPS + 1]
    const float *contrib;
    int32_t V, W;
    float *partial;
    int *err;
};


__global__ void __launch_bounds__(TILE_THREADS, 1) k_tile_gather(TileArgs t) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t slice_bar;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t b = blockIdx.x;
    float *slice = reinterpret_cast<float *>(smem);
    float *stage_base = reinterpret_cast<float *>(smem + slice_bytes(t.W)) + warp * WSTAGE;

    // ---- the block's contributions -> shared memory (bulk copies on one mbarrier) ----
    if (tid == 0) {
        mbar_init(&slice_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
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

    const int2 w0 = t.wtab[(int64_t)b * (TWARPS + 1) + warp];
    const int2 w1 = t.wtab[(int64_t)b * (TWARPS + 1) + warp + 1];
    const int32_t es = w0.x, ee = w1.x;   // edge range of this warp (padded stream positions)
    const int32_t rs = w0.y;              // its first row
    if (es >= ee) return;

    int32_t rowbase = rs;                 // row started by the next head
    float carry = 0.0f;                   // value of the open row (rowbase - 1)
    bool open = false;                    // whether row rowbase-1 belongs to this warp
    const int32_t q_begin = es & ~(WCH - 1);

    // software pipeline: loads of the next chunk are issued before this one is processed
    uint4 nc0, nc1;
    uint32_t nh;
    {
        const int32_t q = q_begin + 16 * lane;
        const uint4 *p = reinterpret_cast<const uint4 *>(t.col16 + q);
        nc0 = __ldg(p);
        nc1 = __ldg(p + 1);
        nh = __ldg(t.heads + (q >> 4));
    }
    for (int32_t q0 = q_begin; q0 < ee; q0 += WCH) {
        const uint4 c0 = nc0, c1 = nc1;
        uint32_t hd = nh;
        if (q0 + WCH < ee) {
            const int32_t q = q0 + WCH + 16 * lane;
            const uint4 *p = reinterpret_cast<const uint4 *>(t.col16 + q);
            nc0 = __ldg(p);
            nc1 = __ldg(p + 1);
            nh = __ldg(t.heads + (q >> 4));
        }
        const uint32_t words[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        float val[16];
        if (q0 >= es && q0 + WCH <= ee) {  // whole chunk inside the warp's range (warp-uniform)
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
    if (open && lane == 0) t.partial[rowbase - 1] = carry;
    if (lane == 0) bulk_store_wait_all();
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

__global__ void k_tile_wtab(const int32_t *rowptr, const int64_t *blk_rows, const int64_t *blk_edges,
                            const int64_t *pbase, int32_t B, int2 *wtab) {
    const int64_t total = (int64_t)B * (TWARPS + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = (int32_t)(t / (TWARPS + 1)), w = (int32_t)(t % (TWARPS + 1));
        const int64_t eb = blk_edges[b], ne = blk_edges[b + 1] - eb;
        const int64_t nominal = eb + (ne * w + TWARPS - 1) / TWARPS;  // global edge index
        int64_t rl = blk_rows[b], rh = blk_rows[b + 1];               // first row starting at >= nominal
        while (rl < rh) {
            const int64_t mid = (rl + rh) >> 1;
            if (rowptr[mid] < nominal) rl = mid + 1; else rh = mid;
        }
        const int64_t edge = (rl < blk_rows[b + 1]) ? rowptr[rl] : blk_edges[b + 1];
        wtab[t] = make_int2((int32_t)(pbase[b] + (edge - eb)), (int32_t)rl);
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
    TC_TRY(p->wtab.alloc((size_t)B * (TWARPS + 1) * 8));
    // grid.y over blocks, grid.x over each block's share: about 8 CTAs per SM in all
    const int gy = B < 65535 ? B : 65535;
    const dim3 grid((unsigned)((sms * 8 + gy - 1) / gy), (unsigned)gy);
    k_tile_copy<<<grid, 256, 0, s>>>(p->colidx.as<int32_t>(), blk_edges.as<int64_t>(), pbase.as<int64_t>(), B, p->W,
                                     p->col16.as<uint16_t>());
    TC_LAUNCH_CHECK();
    k_tile_heads<<<grid, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->blk_rows_dev.as<int64_t>(), blk_edges.as<int64_t>(),
                                      pbase.as<int64_t>(), B, p->heads.as<uint32_t>());
    TC_LAUNCH_CHECK();
    k_tile_wtab<<<(B * (TWARPS + 1) + 255) / 256, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->blk_rows_dev.as<int64_t>(),
                                                               blk_edges.as<int64_t>(), pbase.as<int64_t>(), B,
                                                               p->wtab.as<int2>());
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaStreamSynchronize(s));
    p->padded_edges = npad;
    p->tiled = true;
    return TC_OK;
}

int launch_tiled_gather(const tc_part *p, const float *contrib, int *err_flag, cudaStream_t s, int *launches) {
    const size_t smem = tile_smem_bytes(p->W);
    TC_CUDA(cudaFuncSetAttribute(k_tile_gather, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TileArgs t;
    t.col16 = p->col16.as<uint16_t>();
    t.heads = p->heads.as<uint16_t>();
    t.wtab = p->wtab.as<int2>();
    t.contrib = contrib;
    t.V = p->V;
    t.W = p->W;
    t.partial = const_cast<float *>(p->partial.as<float>());
    t.err = err_flag;
    k_tile_gather<<<p->B, TILE_THREADS, smem, s>>>(t);
    TC_LAUNCH_CHECK();
    ++*launches;
    return TC_OK;
}

}  // namespace tc
