// Graph load: copy and validate an out-edge CSR, build G^T on the device with a stable
// bucket sort by destination (in-rows keep sources ascending), and the out-degree
// reciprocals used by the contribution step of Alg. 1.
#include "tc_internal.cuh"

namespace tc {

__global__ void k_validate_rowptr(const int32_t *rowptr, int32_t V, int64_t E, int *bad) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= V; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = rowptr[v];
        if (v == 0 && a != 0) atomicOr(bad, 1);
        if (v == V && (int64_t)a != E) atomicOr(bad, 2);
        if (v < V && rowptr[v + 1] < a) atomicOr(bad, 4);
    }
}

__global__ void k_validate_colidx(const int32_t *colidx, int64_t E, int32_t V, int *bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = colidx[e];
        if (c < 0 || c >= V) atomicOr(bad, 8);
    }
}

// degree statistics: max in/out degree, dangling count; inv_outdeg = 1/deg (0 if deg == 0)
__global__ void k_degree_stats(const int32_t *out_rowptr, const int32_t *in_rowptr, int32_t V, float *inv_outdeg,
                               int *max_out, int *max_in, unsigned long long *dangling) {
    int lmax_out = 0, lmax_in = 0;
    unsigned long long ldang = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        int od = out_rowptr[v + 1] - out_rowptr[v];
        int id = in_rowptr[v + 1] - in_rowptr[v];
        inv_outdeg[v] = od > 0 ? 1.0f / (float)od : 0.0f;
        lmax_out = max(lmax_out, od);
        lmax_in = max(lmax_in, id);
        ldang += (od == 0);
    }
    for (int d = 16; d > 0; d >>= 1) {
        lmax_out = max(lmax_out, __shfl_down_sync(0xffffffffu, lmax_out, d));
        lmax_in = max(lmax_in, __shfl_down_sync(0xffffffffu, lmax_in, d));
        ldang += __shfl_down_sync(0xffffffffu, ldang, d);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_out, lmax_out);
        atomicMax(max_in, lmax_in);
        atomicAdd(dangling, ldang);
    }
}

static int log2_ceil(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

static int copy_in(void *dst, const void *src, size_t bytes, int mem, cudaStream_t s) {
    if (bytes == 0) return TC_OK;
    TC_CUDA(cudaMemcpyAsync(dst, src, bytes, mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    return TC_OK;
}

static int load_impl(int32_t V, int64_t E, const int32_t *rowptr, const int32_t *colidx, int mem, cudaStream_t s,
                     tc_graph *g) {
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    g->V = V;
    g->E = E;
    g->device = caps.device;
    TC_TRY(g->out_rowptr.alloc(((size_t)V + 1) * 4));
    TC_TRY(g->out_colidx.alloc((size_t)E * 4));
    TC_TRY(g->in_rowptr.alloc(((size_t)V + 1) * 4));
    TC_TRY(g->in_colidx.alloc((size_t)E * 4));
    TC_TRY(g->inv_outdeg.alloc((size_t)V * 4 + 256));  // padded: bulk copies read whole 16-byte units
    TC_TRY(copy_in(g->out_rowptr.p, rowptr, ((size_t)V + 1) * 4, mem, s));
    TC_TRY(copy_in(g->out_colidx.p, colidx, (size_t)E * 4, mem, s));

    DevBuf flags;
    TC_TRY(flags.alloc(64));
    TC_CUDA(cudaMemsetAsync(flags.p, 0, 64, s));
    const int grid = caps.sms * 8;
    k_validate_rowptr<<<grid, 256, 0, s>>>(g->out_rowptr.as<int32_t>(), V, E, flags.as<int>());
    TC_LAUNCH_CHECK();
    k_validate_colidx<<<grid, 256, 0, s>>>(g->out_colidx.as<int32_t>(), E, V, flags.as<int>());
    TC_LAUNCH_CHECK();
    int bad = 0;
    TC_CUDA(cudaMemcpyAsync(&bad, flags.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    if (bad) {
        return fail(TC_ERR_INVALID_GRAPH, "invalid CSR:%s%s%s%s", (bad & 1) ? " rowptr[0]!=0" : "",
                    (bad & 2) ? " rowptr[V]!=E" : "", (bad & 4) ? " rowptr not monotone" : "",
                    (bad & 8) ? " colidx outside [0,V)" : "");
    }

    // G^T: sort (dst, src) pairs by dst, stably; the input is in src order.
    if (E > 0) {
        DevBuf src, kout, ktmp, vtmp;
        TC_TRY(src.alloc((size_t)E * 4));
        TC_TRY(kout.alloc((size_t)E * 4));
        TC_TRY(ktmp.alloc((size_t)E * 4));
        TC_TRY(vtmp.alloc((size_t)E * 4));
        TC_TRY(expand_rows(g->out_rowptr.as<int32_t>(), V, src.as<int32_t>(), s));
        TC_TRY(stable_bucket_sort(g->out_colidx.as<int32_t>(), src.as<int32_t>(), kout.as<int32_t>(),
                                  g->in_colidx.as<int32_t>(), ktmp.as<int32_t>(), vtmp.as<int32_t>(), E, 1,
                                  log2_ceil(V), s));
        TC_TRY(offsets_from_sorted(kout.as<int32_t>(), E, V, g->in_rowptr.as<int32_t>(), s));
        TC_CUDA(cudaStreamSynchronize(s));
    } else {
        TC_CUDA(cudaMemsetAsync(g->in_rowptr.p, 0, ((size_t)V + 1) * 4, s));
    }

    TC_CUDA(cudaMemsetAsync(flags.p, 0, 64, s));
    int *mo = flags.as<int>(), *mi = mo + 1;
    unsigned long long *dg = reinterpret_cast<unsigned long long *>(flags.as<char>() + 8);
    if (V > 0) {
        k_degree_stats<<<grid, 256, 0, s>>>(g->out_rowptr.as<int32_t>(), g->in_rowptr.as<int32_t>(), V,
                                            g->inv_outdeg.as<float>(), mo, mi, dg);
        TC_LAUNCH_CHECK();
    }
    int hs[4] = {0, 0, 0, 0};
    TC_CUDA(cudaMemcpyAsync(hs, flags.p, 16, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    g->max_out_degree = hs[0];
    g->max_in_degree = hs[1];
    unsigned long long nd;
    memcpy(&nd, &hs[2], 8);
    g->num_dangling = (int64_t)nd;
    TC_TRY(collect_hubs(g->in_rowptr.as<int32_t>(), V, g->hub_degree, &g->in_hubs, &g->num_in_hubs, s));
    TC_TRY(collect_hubs(g->out_rowptr.as<int32_t>(), V, g->hub_degree, &g->out_hubs, &g->num_out_hubs, s));
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_graph_load_csr(int32_t V, int64_t E, const int32_t *rowptr, const int32_t *colidx, int mem,
                                 void *stream, tc_graph **out) {
    using namespace tc;
    if (!out) return fail(TC_ERR_INVALID_ARG, "tc_graph_load_csr: out is NULL");
    *out = nullptr;
    if (V < 0 || E < 0) return fail(TC_ERR_INVALID_ARG, "tc_graph_load_csr: negative V or E");
    if ((int64_t)V >= INT32_MAX || E >= INT32_MAX)
        return fail(TC_ERR_UNSUPPORTED, "tc_graph_load_csr: V and E must be < 2^31-1");
    if (!rowptr || (E > 0 && !colidx)) return fail(TC_ERR_INVALID_ARG, "tc_graph_load_csr: null array");
    if (mem != TC_MEM_HOST && mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "tc_graph_load_csr: bad mem flag");
    tc_graph *g = new (std::nothrow) tc_graph();
    if (!g) return fail(TC_ERR_OOM, "tc_graph_load_csr: host allocation failed");
    int st = load_impl(V, E, rowptr, colidx, mem, (cudaStream_t)stream, g);
    if (st != TC_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        delete g;
        return st;
    }
    *out = g;
    return TC_OK;
}

extern "C" void tc_graph_free(tc_graph *g) {
    if (!g) return;
    cudaDeviceSynchronize();
    delete g;
}

extern "C" int tc_graph_get_info(const tc_graph *g, tc_graph_info *info) {
    if (!g || !info) return tc::fail(TC_ERR_INVALID_ARG, "tc_graph_get_info: null argument");
    info->V = g->V;
    info->E = g->E;
    info->max_in_degree = g->max_in_degree;
    info->max_out_degree = g->max_out_degree;
    info->num_dangling = g->num_dangling;
    info->device = g->device;
    return TC_OK;
}

extern "C" int tc_graph_export_transpose(const tc_graph *g, int32_t *rowptr, int32_t *colidx, int mem, void *stream) {
    using namespace tc;
    if (!g) return fail(TC_ERR_INVALID_ARG, "tc_graph_export_transpose: null graph");
    if (mem != TC_MEM_HOST && mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "bad mem flag");
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemcpyKind kind = mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (rowptr) TC_CUDA(cudaMemcpyAsync(rowptr, g->in_rowptr.p, ((size_t)g->V + 1) * 4, kind, s));
    if (colidx && g->E > 0) TC_CUDA(cudaMemcpyAsync(colidx, g->in_colidx.p, (size_t)g->E * 4, kind, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}
