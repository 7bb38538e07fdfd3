// Sparse matrix-vector product y = A x (the SpMV benchmark of Sec. 4, the generalised form of
// the graph operators): A is the CSR loaded as a graph's out-edges (row i = output i), with one
// FP32 value per stored entry in the loaded order.  A warp takes one row at a time: its lanes
// stride the row's entries (coalesced column and value loads, random gathers of x) and a fixed
// shuffle tree adds the 32 lane sums, so the result does not depend on timing.  FP32 throughout.
#include "tc_internal.cuh"

namespace tc {

constexpr int SP_THREADS = 256;

__global__ void __launch_bounds__(SP_THREADS) k_spmv_warp_rows(const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const float *__restrict__ vals,
                                                               const float *__restrict__ x, float *__restrict__ y,
                                                               int32_t nrows) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (SP_THREADS / 32);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrows; r += warps) {
        const int32_t s = __ldg(rowptr + r), e = __ldg(rowptr + r + 1);
        float acc = 0.0f;
        for (int32_t k = s + lane; k < e; k += 32) acc = fmaf(__ldg(vals + k), __ldg(x + __ldg(colidx + k)), acc);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (lane == 0) y[r] = acc;
    }
}

}  // namespace tc

extern "C" int tc_spmv(const tc_graph *g, const float *vals, const float *x, float *y, int mem, void *stream) {
    using namespace tc;
    if (!g || !x || !y || (g->E > 0 && !vals)) return fail(TC_ERR_INVALID_ARG, "tc_spmv: null matrix, values or vector");
    if (mem != TC_MEM_DEVICE && mem != TC_MEM_HOST) return fail(TC_ERR_INVALID_ARG, "tc_spmv: bad mem");
    if (mem != TC_MEM_DEVICE) return fail(TC_ERR_UNSUPPORTED, "tc_spmv: vals, x and y must be device pointers");
    const int32_t V = g->V;
    if (V == 0) return TC_OK;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t want = ((int64_t)V + SP_THREADS / 32 - 1) / (SP_THREADS / 32);
    const int grid = (int)(want < (int64_t)caps.sms * 16 ? want : (int64_t)caps.sms * 16);
    k_spmv_warp_rows<<<grid, SP_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(), vals, x, y,
                                                 V);
    TC_LAUNCH_CHECK();
    return TC_OK;
}
