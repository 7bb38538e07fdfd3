// Device helpers shared by the iteration kernels: block reductions and the
// "last CTA finishes the reduction" pattern used for the dangling rank mass.
#pragma once
#include "tc_internal.cuh"

namespace tc {

// Sum over the block in a fixed tree order (deterministic for a fixed launch shape).
// All threads must call it; the result is valid in every thread.
template <class T>
__device__ __forceinline__ T block_sum(T x, T *smem /* >= 32 entries */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    __syncthreads();
    if (lane == 0) smem[warp] = x;
    __syncthreads();
    T t = 0;
    if (warp == 0) {
        t = lane < nw ? smem[lane] : T(0);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    t = smem[0];
    __syncthreads();
    return t;
}

// Every CTA contributes `mine` (valid in thread 0); the last CTA to arrive sums all the
// contributions in CTA order and stores the total to *out, then re-arms the counter.
__device__ __forceinline__ void grid_sum_last_cta(double mine, double *part, unsigned *counter, double *out) {
    __shared__ bool am_last;
    __shared__ double red[32];
    if (threadIdx.x == 0) {
        part[blockIdx.x] = mine;
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        am_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double t = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) t += __ldcg(part + i);
    t = block_sum<double>(t, red);
    if (threadIdx.x == 0) {
        *out = t;
        *counter = 0u;
    }
}

// Two sums at once (a in x, b in y), same protocol as grid_sum_last_cta.
__device__ __forceinline__ void grid_sum2_last_cta(double a, double b, double *part /* 2 per CTA */,
                                                   unsigned *counter, double *out_a, double *out_b) {
    __shared__ bool am_last2;
    __shared__ double red2[32];
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        am_last2 = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last2) return;
    __threadfence();
    double ta = 0.0, tb = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
        ta += __ldcg(part + 2 * i);
        tb += __ldcg(part + 2 * i + 1);
    }
    ta = block_sum<double>(ta, red2);
    tb = block_sum<double>(tb, red2);
    if (threadIdx.x == 0) {
        *out_a = ta;
        *out_b = tb;
        *counter = 0u;
    }
}

}  // namespace tc
