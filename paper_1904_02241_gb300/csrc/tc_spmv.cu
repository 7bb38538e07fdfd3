// Sparse matrix-vector product y = A x (the SpMV benchmark of Sec. 4, the generalised form of
// the graph operators): A is the CSR loaded as a graph's out-edges (row i = output i), with one
// FP32 value per stored entry in the loaded order.  Rows are mapped the way Sec. 3.2 bins
// them: a group of L lanes per row (L a power of two picked from the mean row length, so a row
// of about 16 entries does not leave 28 of a warp's lanes idle), and a CTA per hub row (more
// than the graph's hub degree, 2048 by default).  Each lane strides its row's entries
// (coalesced column and value loads, random gathers of x) and a fixed shuffle / shared-memory
// tree adds the lane sums, so the result does not depend on timing.  FP32 throughout.
#include "tc_internal.cuh"

namespace tc {

constexpr int SP_THREADS = 256;

template <int L>
__global__ void __launch_bounds__(SP_THREADS) k_spmv_rows(const int32_t *__restrict__ rowptr,
                                                          const int32_t *__restrict__ colidx,
                                                          const float *__restrict__ vals,
                                                          const float *__restrict__ x, float *__restrict__ y,
                                                          int32_t nrows, int32_t hub_degree) {
    constexpr int G = 32 / L;  // rows per warp step
    const int lane = threadIdx.x & 31, sub = lane % L, grp = lane / L;
    const int64_t nw = (int64_t)gridDim.x * (SP_THREADS / 32);
    // every lane runs the same number of steps, so the shuffles below see the whole warp
    for (int64_t base = ((blockIdx.x * (int64_t)SP_THREADS + threadIdx.x) >> 5) * G; base < nrows; base += nw * G) {
        const int64_t r = base + grp;
        int32_t s = 0, e = 0;
        bool mine = false;  // a row of this kernel (not past the end, not a hub row)
        if (r < nrows) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
            mine = e - s <= hub_degree;
            if (!mine) e = s;  // k_spmv_hub
        }
        float acc = 0.0f;
        for (int32_t k = s + sub; k < e; k += L) acc = fmaf(__ldg(vals + k), __ldg(x + __ldg(colidx + k)), acc);
#pragma unroll
        for (int d = L / 2; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
        if (sub == 0 && mine) y[r] = acc;
    }
}

// a CTA per hub row
__global__ void __launch_bounds__(SP_THREADS) k_spmv_hub(const int32_t *__restrict__ rowptr,
                                                         const int32_t *__restrict__ colidx,
                                                         const float *__restrict__ vals, const float *__restrict__ x,
                                                         float *__restrict__ y, const int32_t *__restrict__ hubs) {
    __shared__ float part[SP_THREADS / 32];
    const int32_t r = hubs[blockIdx.x];
    const int32_t s = rowptr[r], e = rowptr[r + 1];
    float acc = 0.0f;
    for (int32_t k = s + threadIdx.x; k < e; k += SP_THREADS) acc = fmaf(__ldg(vals + k), __ldg(x + __ldg(colidx + k)), acc);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < SP_THREADS / 32; ++w) t += part[w];
        y[r] = t;
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
    // lanes per row: the power of two nearest half the mean row length, 4 to 32
    const double mean = (double)g->E / (double)V;
    int L = 4;
    while (L < 32 && 2.0 * L < mean) L *= 2;
    const int64_t want = ((int64_t)V * L + SP_THREADS - 1) / SP_THREADS;
    const int grid = (int)(want < (int64_t)caps.sms * 16 ? (want > 0 ? want : 1) : (int64_t)caps.sms * 16);
    const int32_t *rp = g->out_rowptr.as<int32_t>(), *ci = g->out_colidx.as<int32_t>();
    const int32_t hd = g->hub_degree;
    switch (L) {
        case 4: k_spmv_rows<4><<<grid, SP_THREADS, 0, s>>>(rp, ci, vals, x, y, V, hd); break;
        case 8: k_spmv_rows<8><<<grid, SP_THREADS, 0, s>>>(rp, ci, vals, x, y, V, hd); break;
        case 16: k_spmv_rows<16><<<grid, SP_THREADS, 0, s>>>(rp, ci, vals, x, y, V, hd); break;
        default: k_spmv_rows<32><<<grid, SP_THREADS, 0, s>>>(rp, ci, vals, x, y, V, hd); break;
    }
    TC_LAUNCH_CHECK();
    if (g->num_out_hubs > 0) {
        k_spmv_hub<<<g->num_out_hubs, SP_THREADS, 0, s>>>(rp, ci, vals, x, y, g->out_hubs.as<int32_t>());
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}
