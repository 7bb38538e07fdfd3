// Device helpers shared by the iteration kernels: block reductions and the
// "last CTA finishes the reduction" pattern used for the dangling rank mass.
#pragma once
#include "tc_internal.cuh"

namespace tc {

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

// Programmatic dependent launch: a kernel launched with the programmatic stream serialization
// attribute may start while the previous kernel in the stream finishes; pdl_wait() blocks until
// that kernel has completed and its writes are visible (a no-op without the attribute), and
// pdl_trigger() lets the next kernel start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


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
// contributions in CTA order and stores the total plus `extra` to *out, then re-arms the counter.
__device__ __forceinline__ void grid_sum_last_cta(double mine, double *part, unsigned *counter, double *out,
                                                  double extra = 0.0) {
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
        *out = t + extra;
        *counter = 0u;
    }
}

// Every CTA has written its share into slots of part[0, nslots) (any CTA any slot); the last
// CTA to arrive sums the slots in slot order (deterministic whichever CTA filled which slot),
// stores the total to *out and re-arms the counter and *queue (a work queue the CTAs drew from,
// idle by now: every CTA drew its last item before arriving).  All threads must call it.
__device__ __forceinline__ void grid_sum_slots_last_cta(const double *part, int32_t nslots, unsigned *counter,
                                                        unsigned *queue, double *out, double extra = 0.0) {
    __shared__ bool am_last3;
    __shared__ double red3[32];
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        am_last3 = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last3) return;
    __threadfence();
    double t = 0.0;
    for (int32_t i = threadIdx.x; i < nslots; i += blockDim.x) t += __ldcg(part + i);
    t = block_sum<double>(t, red3);
    if (threadIdx.x == 0) {
        *out = t + extra;
        *counter = 0u;
        *queue = 0u;
    }
}

// Two sums at once (a in x, b in y), same protocol as grid_sum_last_cta.
// Returns true in every thread of the last CTA (after the sums are written).
__device__ __forceinline__ bool grid_sum2_last_cta(double a, double b, double *part /* 2 per CTA */,
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
    if (!am_last2) return false;
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
    return true;
}

}  // namespace tc
