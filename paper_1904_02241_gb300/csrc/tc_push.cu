// Staged push scatter: Alg. 5 with each block's destination range held in shared memory.
//
// A TC_PUSH partition cuts the destinations into ranges of W vertices (Sec. 3.1, Fig. 3 with
// the roles of rows and columns swapped); the paper keeps a block's range of `sums` resident in
// L2 and adds every edge's contribution there with a global atomic.  When the range fits in
// shared memory (W * 8 bytes), a CTA instead adds a slice of the block's edges into a shared
// copy of the range and then adds each nonzero sum of the copy to global memory once: the
// per-edge reductions become shared-memory atomics, and the global ones drop from one per edge
// to at most one per destination per CTA.
//
// Sums are 64-bit fixed-point integers (exact in any order, so the ranks repeat bit for bit) or,
// in the paper's form, FP32 (order-dependent rounding).
#include <algorithm>
#include <vector>

#include "tc_common_dev.cuh"

namespace tc {

constexpr int PS_THREADS = 1024;

// Widest destination range whose 8-byte sums fit one CTA's shared memory (a multiple of 32).
int32_t push_smem_width(int max_smem_optin) {
    int64_t W = ((int64_t)max_smem_optin - 1024) / 8;
    W = W / 32 * 32;
    return W > 0 ? (int32_t)W : 0;
}

// round(y) as a 64-bit two's-complement integer for |y| < 2^62, from the FP32 bits.
__device__ __forceinline__ unsigned long long ps_round64(float y) {
    const uint32_t b = __float_as_uint(y);
    const uint32_t a = b & 0x7fffffffu;
    const int e = (int)(a >> 23);
    const unsigned long long m = (a & 0x7fffffu) | (e ? 0x800000u : 0u);
    const int sh = (e ? e : 1) - 150;  // |y| = m * 2^sh
    unsigned long long r;
    if (sh >= 0) r = m << sh;
    else if (sh <= -25) r = 0ull;
    else r = (m + (1ull << (-sh - 1))) >> (-sh);
    return (b >> 31) ? (0ull - r) : r;
}

// One CTA per tile (block b, edges [e0, e1)): shared sums of the block's range, then one global
// addition per nonzero entry.  scalef: the fixed-point scale (FIXED only).
template <bool FIXED>
__global__ void __launch_bounds__(PS_THREADS, 1) k_push_smem(const int4 *__restrict__ tiles,
                                                             const int32_t *__restrict__ esrc,
                                                             const int32_t *__restrict__ dst, int32_t W, int32_t V,
                                                             const float *__restrict__ contrib, void *sums,
                                                             const double *fx_scale) {
    extern __shared__ __align__(16) unsigned char psm[];
    unsigned long long *acc64 = reinterpret_cast<unsigned long long *>(psm);
    float *acc32 = reinterpret_cast<float *>(psm);
    const int4 t = tiles[blockIdx.x];
    const int64_t lo = (int64_t)t.x * W;
    const int32_t w = (int32_t)(((int64_t)V - lo) < W ? ((int64_t)V - lo) : W);
    const int64_t e0 = ((int64_t)t.z << 31) | (uint32_t)t.y;  // 62-bit edge bounds split in two ints
    const int64_t e1 = e0 + (uint32_t)t.w;
    const float scalef = FIXED ? (float)(*fx_scale * 0x1p-6) : 1.0f;  // |sum| < 2^55
    for (int32_t v = threadIdx.x; v < w; v += PS_THREADS) {
        if (FIXED) acc64[v] = 0ull;
        else acc32[v] = 0.0f;
    }
    __syncthreads();
    int64_t i = e0 + threadIdx.x;
    for (; i + 3 * PS_THREADS < e1; i += 4 * PS_THREADS) {  // four edges in flight per thread
        int32_t sv[4], dv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sv[k] = __ldg(esrc + i + k * PS_THREADS);
            dv[k] = (int32_t)(__ldg(dst + i + k * PS_THREADS) - lo);
        }
        float cv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cv[k] = __ldg(contrib + sv[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (cv[k] == 0.0f) continue;
            if (FIXED) atomicAdd(acc64 + dv[k], ps_round64(cv[k] * scalef));
            else atomicAdd(acc32 + dv[k], cv[k]);
        }
    }
    for (; i < e1; i += PS_THREADS) {
        const float c = __ldg(contrib + __ldg(esrc + i));
        if (c == 0.0f) continue;
        const int32_t d = (int32_t)(__ldg(dst + i) - lo);
        if (FIXED) atomicAdd(acc64 + d, ps_round64(c * scalef));
        else atomicAdd(acc32 + d, c);
    }
    __syncthreads();
    for (int32_t v = threadIdx.x; v < w; v += PS_THREADS) {
        if (FIXED) {
            const unsigned long long x = acc64[v];
            if (x) atomicAdd(static_cast<unsigned long long *>(sums) + lo + v, x);
        } else {
            const float x = acc32[v];
            if (x != 0.0f) atomicAdd(static_cast<float *>(sums) + lo + v, x);
        }
    }
}

// Tiles of the staged push: block b's edges cut into n_b = max(1, round(E_b / T)) equal slices,
// T = E / (three waves of one CTA per SM); the largest blocks' tiles first.
int build_push_tiles(tc_part *p, int sms, cudaStream_t s) {
    p->nptiles = 0;
    if (p->E == 0) return TC_OK;
    TC_CUDA(cudaStreamSynchronize(s));  // the host copies of the block bounds
    const int64_t T = p->E / (3LL * sms) > 0 ? p->E / (3LL * sms) : 1;
    std::vector<int4> h;
    std::vector<int64_t> cost;
    for (int32_t b = 0; b < p->B; ++b) {
        const int64_t eb = p->h_blk_edges[b + 1] - p->h_blk_edges[b];
        if (eb == 0) continue;
        int64_t n = (eb + T / 2) / T;
        if (n < 1) n = 1;
        for (int64_t k = 0; k < n; ++k) {
            const int64_t a = p->h_blk_edges[b] + eb * k / n, z = p->h_blk_edges[b] + eb * (k + 1) / n;
            if (z - a > INT32_MAX) return fail(TC_ERR_UNSUPPORTED, "build_push_tiles: a tile over 2^31 edges");
            h.push_back(make_int4(b, (int32_t)(a & 0x7fffffff), (int32_t)(a >> 31), (int32_t)(z - a)));
            cost.push_back(z - a);
        }
    }
    std::vector<int32_t> order(h.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int32_t)i;
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return cost[x] > cost[y]; });
    std::vector<int4> hs(h.size());
    for (size_t i = 0; i < order.size(); ++i) hs[i] = h[(size_t)order[i]];
    TC_TRY(p->ptiles.alloc(hs.size() * sizeof(int4)));
    TC_CUDA(cudaMemcpyAsync(p->ptiles.p, hs.data(), hs.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    TC_CUDA(cudaStreamSynchronize(s));  // hs is freed at return
    p->nptiles = (int32_t)hs.size();
    return TC_OK;
}

int launch_push_smem(const tc_part *p, const float *contrib, void *sums, const double *fx_scale, bool fixed,
                     cudaStream_t s) {
    if (p->nptiles == 0) return TC_OK;
    const size_t smem = (size_t)p->W * (fixed ? 8 : 4);
    const void *k = fixed ? (const void *)k_push_smem<true> : (const void *)k_push_smem<false>;
    TC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (fixed)
        k_push_smem<true><<<p->nptiles, PS_THREADS, smem, s>>>(p->ptiles.as<int4>(), p->esrc.as<int32_t>(),
                                                               p->colidx.as<int32_t>(), p->W, p->V, contrib, sums,
                                                               fx_scale);
    else
        k_push_smem<false><<<p->nptiles, PS_THREADS, smem, s>>>(p->ptiles.as<int4>(), p->esrc.as<int32_t>(),
                                                                p->colidx.as<int32_t>(), p->W, p->V, contrib, sums,
                                                                fx_scale);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace tc
