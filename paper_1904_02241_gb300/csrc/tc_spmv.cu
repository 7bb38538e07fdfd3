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

// ---------------------------------------------------------------------------------------------
// GC-pull SpMV (Sec. 4's SpMV with TOCAB, a value stream of 4 B per entry): a TC_PUSH partition
// of the matrix's CSR cuts its columns into ranges of W (so x[block] is the block's working set,
// Sec. 3.1 with the value read from x instead of the contributions); each (block, row) piece is a
// local row whose partial sum goes to partial[], and the merge of Fig. 5 adds a row's pieces in
// block order into y.  FP32; deterministic (a fixed order everywhere).
// ---------------------------------------------------------------------------------------------
namespace tc {

__global__ void k_iota(int64_t n, int32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (int32_t)i;
}

__global__ void k_gather_vals(const int32_t *__restrict__ perm, const float *__restrict__ vals, int64_t n,
                              float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = vals[perm[i]];
}

// Local rows: a lane each below 32 entries (in order), a warp each from 32 (lane strides in
// order, then a fixed shuffle tree).
__global__ void __launch_bounds__(SP_THREADS) k_spmv_block_rows(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx,
                                                                const float *__restrict__ pvals,
                                                                const float *__restrict__ x, int64_t R,
                                                                float *__restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (SP_THREADS / 32);
    for (int64_t grp = (blockIdx.x * (int64_t)SP_THREADS + threadIdx.x) >> 5; grp * 32 < R; grp += nw) {
        const int64_t r = grp * 32 + lane;
        int32_t s = 0, e = 0;
        if (r < R) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
        }
        float acc = 0.0f;
        if (e - s < 32)
            for (int32_t k = s; k < e; ++k) acc = fmaf(__ldg(pvals + k), __ldg(x + __ldg(colidx + k)), acc);
        unsigned long_rows = __ballot_sync(0xffffffffu, e - s >= 32);
        while (long_rows) {
            const int l = __ffs(long_rows) - 1;
            long_rows &= long_rows - 1;
            const int32_t ls = __shfl_sync(0xffffffffu, s, l), le = __shfl_sync(0xffffffffu, e, l);
            float w = 0.0f;
            for (int32_t k = ls + lane; k < le; k += 32) w = fmaf(__ldg(pvals + k), __ldg(x + __ldg(colidx + k)), w);
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
            if (lane == l) acc = w;
        }
        if (r < R) partial[r] = acc;
    }
}

// Fig. 5: CTA j owns rows [j k, (j+1) k); it adds block b's slice for b = 0, 1, ... in order (the
// rows of one slice are distinct, so its threads never collide), then writes y.
__global__ void __launch_bounds__(SP_THREADS) k_spmv_merge(const float *__restrict__ partial,
                                                           const int32_t *__restrict__ id_map,
                                                           const int32_t *__restrict__ merge_off, int32_t B,
                                                           int32_t nranges, int32_t k, int32_t V, float *y) {
    extern __shared__ float macc[];  // [k]
    for (int32_t j = blockIdx.x; j < nranges; j += gridDim.x) {
        const int32_t vbase = j * k;
        for (int32_t t = threadIdx.x; t < k; t += SP_THREADS) macc[t] = 0.0f;
        __syncthreads();
        for (int32_t b = 0; b < B; ++b) {
            const int32_t *o = merge_off + (int64_t)b * (nranges + 1) + j;
            const int32_t r0 = __ldg(o), r1 = __ldg(o + 1);
            for (int32_t r = r0 + threadIdx.x; r < r1; r += SP_THREADS) macc[__ldg(id_map + r) - vbase] += __ldg(partial + r);
            __syncthreads();
        }
        for (int32_t t = threadIdx.x; t < k && vbase + t < V; t += SP_THREADS) y[vbase + t] = macc[t];
        __syncthreads();
    }
}

// GC-push (Sec. 4's SpMV in the push direction with TOCAB): the pieces of a TC_PULL partition of
// the matrix's graph.  Piece r = (row block b, column j = id_map[r]) holds the entries (i, j) of
// A with i in block b; x[j] is read once per piece and every entry adds vals * x[j] into y[i]
// with an FP32 atomic add.  The pieces are stored block after block, so while a block's pieces
// run, the atomics land in its W-entry slice of y, which the L2 holds (Sec. 3.1 with y as the
// working set).  Load balancing as Sec. 3.2 bins it: a lane per piece below 32 entries, a warp
// per longer one.  The order of the additions into y[i] depends on timing.
__global__ void __launch_bounds__(SP_THREADS) k_spmv_push_pieces(const int32_t *__restrict__ rowptr,
                                                                 const int32_t *__restrict__ colidx,
                                                                 const float *__restrict__ pvals,
                                                                 const int32_t *__restrict__ id_map,
                                                                 const float *__restrict__ x, int64_t R, float *y) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (SP_THREADS / 32);
    for (int64_t grp = (blockIdx.x * (int64_t)SP_THREADS + threadIdx.x) >> 5; grp * 32 < R; grp += nw) {
        const int64_t r = grp * 32 + lane;
        int32_t s = 0, e = 0;
        float xj = 0.0f;
        if (r < R) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
            xj = __ldg(x + __ldg(id_map + r));
        }
        if (e - s < 32)
            for (int32_t k = s; k < e; ++k) atomicAdd(y + __ldg(colidx + k), __ldg(pvals + k) * xj);
        unsigned long_rows = __ballot_sync(0xffffffffu, e - s >= 32);
        while (long_rows) {
            const int l = __ffs(long_rows) - 1;
            long_rows &= long_rows - 1;
            const int32_t ls = __shfl_sync(0xffffffffu, s, l), le = __shfl_sync(0xffffffffu, e, l);
            const float xl = __shfl_sync(0xffffffffu, xj, l);
            for (int32_t k = ls + lane; k < le; k += 32) atomicAdd(y + __ldg(colidx + k), __ldg(pvals + k) * xl);
        }
    }
}

}  // namespace tc

extern "C" int tc_part_set_values(tc_part *p, const float *vals, int mem, void *stream) {
    using namespace tc;
    if (!p || (p->E > 0 && !vals)) return fail(TC_ERR_INVALID_ARG, "tc_part_set_values: null partition or values");
    if (p->dir != TC_PUSH && p->dir != TC_PULL) return fail(TC_ERR_INVALID_ARG, "tc_part_set_values: bad partition");
    if (p->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_part_set_values: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if (mem != TC_MEM_DEVICE) return fail(TC_ERR_UNSUPPORTED, "tc_part_set_values: vals must be a device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t E = p->E;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    const int grid = caps.sms * 8;
    if (!p->pperm_built) {  // the partition's own sorts again, carrying each entry's position
        TC_TRY(p->pperm.alloc((size_t)(E > 0 ? E : 1) * 4));
        if (E > 0) {
            DevBuf iota, keys, kt, vt, tpos;
            TC_TRY(iota.alloc((size_t)E * 4));
            k_iota<<<grid, 256, 0, s>>>(E, iota.as<int32_t>());
            TC_LAUNCH_CHECK();
            TC_TRY(keys.alloc((size_t)E * 4));
            TC_TRY(kt.alloc((size_t)E * 4));
            TC_TRY(vt.alloc((size_t)E * 4));
            // the entries in the order the partition's stream starts from: the CSR itself for a
            // push partition; for a pull partition G^T, the graph load's stable sort by column
            const int32_t *ci = p->g->out_colidx.as<int32_t>();
            const int32_t *pos = iota.as<int32_t>();
            if (p->dir == TC_PULL) {
                int vbits = 0;
                while ((1LL << vbits) < (int64_t)p->V) ++vbits;
                TC_TRY(tpos.alloc((size_t)E * 4));
                TC_TRY(stable_bucket_sort(ci, iota.as<int32_t>(), keys.as<int32_t>(), tpos.as<int32_t>(),
                                          kt.as<int32_t>(), vt.as<int32_t>(), E, 1, vbits, s));
                ci = p->g->in_colidx.as<int32_t>();
                pos = tpos.as<int32_t>();
            }
            if (p->B > 1) {
                int bits = 0;
                while ((1LL << bits) < (int64_t)p->B) ++bits;
                TC_TRY(stable_bucket_sort(ci, pos, keys.as<int32_t>(), p->pperm.as<int32_t>(), kt.as<int32_t>(),
                                          vt.as<int32_t>(), E, p->W, bits, s));
            } else {
                TC_CUDA(cudaMemcpyAsync(p->pperm.p, pos, (size_t)E * 4, cudaMemcpyDeviceToDevice, s));
            }
            TC_CUDA(cudaStreamSynchronize(s));  // the scratch is freed at the end of this block
        }
        p->pperm_built = true;
    }
    TC_TRY(p->pvals.alloc((size_t)(E > 0 ? E : 1) * 4));
    if (E > 0) {
        k_gather_vals<<<grid, 256, 0, s>>>(p->pperm.as<int32_t>(), vals, E, p->pvals.as<float>());
        TC_LAUNCH_CHECK();
    }
    TC_CUDA(cudaStreamSynchronize(s));
    p->has_vals = true;
    return TC_OK;
}

extern "C" int tc_spmv_tocab(const tc_part *p, const float *x, float *y, int mem, void *stream) {
    using namespace tc;
    if (!p || !x || !y) return fail(TC_ERR_INVALID_ARG, "tc_spmv_tocab: null partition or vector");
    if (!p->has_vals)
        return fail(TC_ERR_INVALID_ARG, "tc_spmv_tocab: needs a partition given values by tc_part_set_values");
    if (mem != TC_MEM_DEVICE) return fail(TC_ERR_UNSUPPORTED, "tc_spmv_tocab: x and y must be device pointers");
    const int32_t V = p->V;
    if (V == 0) return TC_OK;
    if (p->dir == TC_PULL) {  // GC-push: y = 0, then the pieces add into it
        DeviceCaps caps;
        TC_TRY(device_caps(&caps));
        cudaStream_t s = (cudaStream_t)stream;
        TC_CUDA(cudaMemsetAsync(y, 0, (size_t)V * 4, s));
        if (p->R > 0) {
            const int64_t want = (p->R + SP_THREADS - 1) / SP_THREADS;
            const int grid = (int)(want < (int64_t)caps.sms * 16 ? want : (int64_t)caps.sms * 16);
            k_spmv_push_pieces<<<grid, SP_THREADS, 0, s>>>(p->rowptr.as<int32_t>(), p->colidx.as<int32_t>(),
                                                           p->pvals.as<float>(), p->id_map.as<int32_t>(), x, p->R, y);
            TC_LAUNCH_CHECK();
        }
        return TC_OK;
    }
    if ((size_t)p->k * 4 > 200 * 1024) return fail(TC_ERR_UNSUPPORTED, "tc_spmv_tocab: merge_range above 51,200");
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    cudaStream_t s = (cudaStream_t)stream;
    if (p->R > 0) {
        const int64_t want = (p->R + SP_THREADS - 1) / SP_THREADS;
        const int grid = (int)(want < (int64_t)caps.sms * 16 ? (want > 0 ? want : 1) : (int64_t)caps.sms * 16);
        k_spmv_block_rows<<<grid, SP_THREADS, 0, s>>>(p->rowptr.as<int32_t>(), p->colidx.as<int32_t>(),
                                                      p->pvals.as<float>(), x, p->R,
                                                      const_cast<float *>(p->partial.as<float>()));
        TC_LAUNCH_CHECK();
    }
    const size_t smem = (size_t)p->k * 4;
    TC_CUDA(cudaFuncSetAttribute(k_spmv_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int mgrid = p->nranges < caps.sms * 8 ? (p->nranges > 0 ? p->nranges : 1) : caps.sms * 8;
    k_spmv_merge<<<mgrid, SP_THREADS, smem, s>>>(p->partial.as<float>(), p->id_map.as<int32_t>(),
                                                 p->merge_off.as<int32_t>(), p->B, p->nranges, p->k, V, y);
    TC_LAUNCH_CHECK();
    return TC_OK;
}
