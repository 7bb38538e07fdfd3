// Betweenness centrality (the traversal benchmark of Sec. 3.3 and Sec. 4).
//
// Forward sweep: the shortest-path calculation of Alg. 3 (depth delta and shortest-path count
// sigma from one source), run topology-driven in the pull direction over G^T: in level L every
// vertex not yet reached adds up sigma over its in-neighbours of depth L, and takes depth L+1 if
// it has any.  Pull needs no atomics (a vertex is written only by its own thread) and sums in
// in-row order, so it is deterministic.  A thread reads depth[u] of in-neighbours that other
// threads may set to L+1 in the same launch; both the old value (-1) and the new one differ from
// L, so the read is unaffected, and sigma[u] is read only for vertices of depth L, which no one
// writes in this level.
//
// Backward sweep: the dependency back-propagation of the BC the paper cites, pulled over the
// out-edges of G level by level from the deepest: for a vertex v of depth L,
//   dep[v] = sum over out-neighbours w of depth L+1 of sigma[v] / sigma[w] * (1 + dep[w]),
// in out-row order, and every vertex other than the source adds dep[v] to its score.  The
// products, quotients and sums are rounded one by one (no fused multiply-add), in the order of
// that formula.
//
// sigma, dep and the scores are FP64 (sigma is an integer count, exact below 2^53).
#include "tc_internal.cuh"

namespace tc {

constexpr int BC_THREADS = 256;

__global__ void k_bc_init(int32_t V, int32_t source, int32_t *depth, double *sigma, double *dep) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        depth[v] = v == source ? 0 : -1;
        sigma[v] = v == source ? 1.0 : 0.0;
        dep[v] = 0.0;
    }
}

__global__ void k_bc_zero(int32_t V, double *score) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        score[v] = 0.0;
}

// level L -> L+1 of Alg. 3 in pull form; *found counts the vertices reached
__global__ void __launch_bounds__(BC_THREADS) k_bc_forward(const int32_t *__restrict__ in_rowptr,
                                                           const int32_t *__restrict__ in_colidx, int32_t V,
                                                           int32_t L, int32_t *depth, double *sigma,
                                                           unsigned *found) {
    unsigned n = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        if (depth[v] != -1) continue;
        double acc = 0.0;
        bool hit = false;
        for (int32_t e = in_rowptr[v]; e < in_rowptr[v + 1]; ++e) {
            const int32_t u = in_colidx[e];
            if (depth[u] == L) {
                acc = __dadd_rn(acc, sigma[u]);
                hit = true;
            }
        }
        if (hit) {
            depth[v] = L + 1;
            sigma[v] = acc;
            ++n;
        }
    }
    if (n) atomicAdd(found, n);
}

// dependencies of the vertices of depth L (those of depth L+1 are final)
__global__ void __launch_bounds__(BC_THREADS) k_bc_backward(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx, int32_t V,
                                                            int32_t L, int32_t source,
                                                            const int32_t *__restrict__ depth,
                                                            const double *__restrict__ sigma, double *dep,
                                                            double *score) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        if (depth[v] != L) continue;
        const double sv = sigma[v];
        double d = 0.0;
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            const int32_t w = colidx[e];
            if (depth[w] == L + 1) d = __dadd_rn(d, __dmul_rn(__ddiv_rn(sv, sigma[w]), __dadd_rn(1.0, dep[w])));
        }
        dep[v] = d;
        if (v != source) score[v] = __dadd_rn(score[v], d);
    }
}

// Forward sweep from `source` into depth/sigma (device); returns the deepest level reached.
static int bc_forward_impl(const tc_graph *g, int32_t source, int32_t *depth, double *sigma, double *dep,
                           unsigned *found_dev, unsigned *found_host, int grid, cudaStream_t s, int32_t *max_depth) {
    const int32_t V = g->V;
    k_bc_init<<<grid, BC_THREADS, 0, s>>>(V, source, depth, sigma, dep);
    TC_LAUNCH_CHECK();
    int32_t L = 0;
    for (;; ++L) {
        TC_CUDA(cudaMemsetAsync(found_dev, 0, 4, s));
        k_bc_forward<<<grid, BC_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), V, L,
                                                 depth, sigma, found_dev);
        TC_LAUNCH_CHECK();
        TC_CUDA(cudaMemcpyAsync(found_host, found_dev, 4, cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        if (*found_host == 0) break;
    }
    *max_depth = L;
    return TC_OK;
}

struct BcScratch {
    DevBuf depth, sigma, dep, score, found;
    unsigned found_host = 0;
    int grid = 1;
    int setup(int32_t V, bool need_score) {
        DeviceCaps caps;
        TC_TRY(device_caps(&caps));
        grid = caps.sms * 8;
        TC_TRY(depth.alloc((size_t)V * 4));
        TC_TRY(sigma.alloc((size_t)V * 8));
        TC_TRY(dep.alloc((size_t)V * 8));
        if (need_score) TC_TRY(score.alloc((size_t)V * 8));
        TC_TRY(found.alloc(16));
        return TC_OK;
    }
};

}  // namespace tc

extern "C" int tc_bc_forward(const tc_graph *g, int32_t source, int out_mem, int32_t *depth_out, double *sigma_out,
                             void *stream) {
    using namespace tc;
    if (!g || !depth_out || !sigma_out) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: null graph or output");
    if (source < 0 || source >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: source outside [0, V)");
    if (out_mem != TC_MEM_HOST && out_mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "tc_bc_forward: bad out_mem");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t V = g->V;
    BcScratch w;
    TC_TRY(w.setup(V, false));
    int32_t maxd = 0;
    TC_TRY(bc_forward_impl(g, source, w.depth.as<int32_t>(), w.sigma.as<double>(), w.dep.as<double>(),
                           w.found.as<unsigned>(), &w.found_host, w.grid, s, &maxd));
    const cudaMemcpyKind kind = out_mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    TC_CUDA(cudaMemcpyAsync(depth_out, w.depth.p, (size_t)V * 4, kind, s));
    TC_CUDA(cudaMemcpyAsync(sigma_out, w.sigma.p, (size_t)V * 8, kind, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

extern "C" int tc_bc(const tc_graph *g, const int32_t *sources, int32_t num_sources, int out_mem, double *scores_out,
                     void *stream) {
    using namespace tc;
    if (!g || !scores_out || (num_sources > 0 && !sources))
        return fail(TC_ERR_INVALID_ARG, "tc_bc: null graph, sources or output");
    if (num_sources < 0) return fail(TC_ERR_INVALID_ARG, "tc_bc: num_sources < 0");
    if (out_mem != TC_MEM_HOST && out_mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "tc_bc: bad out_mem");
    for (int32_t k = 0; k < num_sources; ++k)
        if (sources[k] < 0 || sources[k] >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_bc: a source is outside [0, V)");
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t V = g->V;
    if (V == 0) return TC_OK;
    BcScratch w;
    const bool dev_out = out_mem == TC_MEM_DEVICE;
    TC_TRY(w.setup(V, !dev_out));
    double *score = dev_out ? scores_out : w.score.as<double>();
    k_bc_zero<<<w.grid, BC_THREADS, 0, s>>>(V, score);
    TC_LAUNCH_CHECK();
    for (int32_t k = 0; k < num_sources; ++k) {
        int32_t maxd = 0;
        TC_TRY(bc_forward_impl(g, sources[k], w.depth.as<int32_t>(), w.sigma.as<double>(), w.dep.as<double>(),
                               w.found.as<unsigned>(), &w.found_host, w.grid, s, &maxd));
        for (int32_t L = maxd; L >= 0; --L) {
            k_bc_backward<<<w.grid, BC_THREADS, 0, s>>>(g->out_rowptr.as<int32_t>(), g->out_colidx.as<int32_t>(), V, L,
                                                        sources[k], w.depth.as<int32_t>(), w.sigma.as<double>(),
                                                        w.dep.as<double>(), score);
            TC_LAUNCH_CHECK();
        }
    }
    if (!dev_out) TC_CUDA(cudaMemcpyAsync(scores_out, score, (size_t)V * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}
