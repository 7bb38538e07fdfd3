// tc_pagerank_pull_noalloc: unblocked pull PageRank that allocates no memory.
//
// For callers that must not allocate device memory: for example a plug-in running inside
// a host framework whose allocator owns the whole device memory pool, or a service that
// fixes its memory budget at start-up and forbids cudaMalloc/cudaFree afterwards.  Such a
// caller passes its device-resident in-edge CSR, out-degrees and output buffer; the
// iteration's scratch (contributions, out-degree reciprocals, dangling-mass partials) lives
// in the file-scope device array below, which every GPU that loads this library holds
// until the process exits.  Under CUDA's default lazy module loading that array is reserved
// on a device when this module is first used there, i.e. by the first call of the entry
// point on that device; a caller whose memory budget is fixed later should make that first
// call at start-up (or load modules eagerly with CUDA_MODULE_LOADING=EAGER).
#include <mutex>

#include "tc_common_dev.cuh"

namespace tc {
namespace noalloc {

constexpr int THREADS = 256;
constexpr int WARPS = THREADS / 32;
constexpr int64_t MAX_V = TC_NOALLOC_MAX_V;
constexpr int64_t MAX_CTAS = 4096;                       // capacity of the per-CTA partials
constexpr size_t HEAD_BYTES = 256;                       // D[2] doubles + arrival counter
constexpr size_t PART_BYTES = (size_t)MAX_CTAS * 8;      // per-CTA dangling partials
constexpr size_t VEC_BYTES = (size_t)MAX_V * 4;          // one float per vertex
constexpr size_t SCRATCH_BYTES = HEAD_BYTES + PART_BYTES + 3 * VEC_BYTES;
static_assert(SCRATCH_BYTES == TC_NOALLOC_SCRATCH_BYTES, "header and implementation disagree");

// The scratch.  Host code must not pass this symbol to a kernel: on the host it names a
// stand-in, not device memory.  Its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

struct Layout {
    double *D;           // D[0], D[1]: dangling mass, ping-pong between iterations
    unsigned *counter;   // arrival counter of the last-CTA reduction (must start at 0)
    double *dpart;       // [MAX_CTAS]
    float *contrib[2];   // [MAX_V] each
    float *inv_outdeg;   // [MAX_V]
};

static Layout layout(unsigned char *base) {
    Layout l;
    l.D = reinterpret_cast<double *>(base);
    l.counter = reinterpret_cast<unsigned *>(base + 32);
    l.dpart = reinterpret_cast<double *>(base + HEAD_BYTES);
    l.contrib[0] = reinterpret_cast<float *>(base + HEAD_BYTES + PART_BYTES);
    l.contrib[1] = l.contrib[0] + MAX_V;
    l.inv_outdeg = l.contrib[1] + MAX_V;
    return l;
}

// Initial ranks 1/V, first contributions, reciprocals of the caller's out-degrees and the
// dangling mass of the initial ranks.
__global__ void __launch_bounds__(THREADS) k_init(int32_t V, const int32_t *__restrict__ out_degree, Layout l,
                                                  float *rank_out) {
    __shared__ float fred[32];
    float dsum = 0.0f;
    const float r0 = 1.0f / (float)V;
    for (int64_t v = blockIdx.x * (int64_t)THREADS + threadIdx.x; v < V; v += (int64_t)gridDim.x * THREADS) {
        const int32_t od = out_degree[v];
        const float inv = od > 0 ? 1.0f / (float)od : 0.0f;
        l.inv_outdeg[v] = inv;
        l.contrib[0][v] = r0 * inv;
        if (rank_out) rank_out[v] = r0;
        if (od == 0) dsum += r0;
    }
    const float bs = block_sum<float>(dsum, fred);
    grid_sum_last_cta((double)bs, l.dpart, l.counter, l.D + 0);
}

// One Jacobi iteration of Alg. 1 with the update fused: a warp takes 32 consecutive
// destinations; rows under 32 edges are summed by their lane, longer rows by the warp.
__global__ void __launch_bounds__(THREADS) k_gather(const int32_t *__restrict__ rowptr,
                                                    const int32_t *__restrict__ colidx, int32_t V, Layout l, int cur,
                                                    float base, float damping, int drop, float *rank_out) {
    __shared__ float fred[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float *__restrict__ contrib = l.contrib[cur];
    float *contrib_next = l.contrib[cur ^ 1];
    const float spread = drop ? 0.0f : (float)(l.D[cur] / (double)V);
    float dsum = 0.0f;
    const int64_t ngroups = ((int64_t)V + 31) >> 5;
    for (int64_t grp = (int64_t)blockIdx.x * WARPS + warp; grp < ngroups; grp += (int64_t)gridDim.x * WARPS) {
        const int64_t v = grp * 32 + lane;
        const bool valid = v < V;
        int32_t s = 0, e = 0;
        if (valid) {
            s = __ldg(rowptr + v);
            e = __ldg(rowptr + v + 1);
        }
        const int32_t deg = e - s;
        float sum = 0.0f;
        if (deg < 32)
            for (int32_t i = s; i < e; ++i) sum += contrib[__ldg(colidx + i)];
        unsigned wm = __ballot_sync(0xffffffffu, valid && deg >= 32);
        while (wm) {
            const int ln = __ffs(wm) - 1;
            wm &= wm - 1;
            const int32_t ws = __shfl_sync(0xffffffffu, s, ln), we = __shfl_sync(0xffffffffu, e, ln);
            float acc = 0.0f;
            // 64-bit index: ws + lane + 32 k may pass INT32_MAX when a row ends near 2^31 - 1
            for (int64_t i = (int64_t)ws + lane; i < we; i += 32) acc += contrib[__ldg(colidx + i)];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
            if (lane == ln) sum = acc;
        }
        if (valid) {
            const float r = base + damping * (sum + spread);
            if (rank_out) rank_out[v] = r;
            const float inv = l.inv_outdeg[v];
            contrib_next[v] = r * inv;
            if (inv == 0.0f) dsum += r;
        }
    }
    const float bs = block_sum<float>(dsum, fred);
    grid_sum_last_cta((double)bs, l.dpart, l.counter, l.D + (cur ^ 1));
}

// Device address of g_scratch for the current device, looked up once per device.
static int scratch_address(unsigned char **out) {
    static std::mutex mtx;
    static void *addr[256] = {nullptr};
    int dev = 0;
    TC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(TC_ERR_UNSUPPORTED, "tc_pagerank_pull_noalloc: device index %d", dev);
    std::lock_guard<std::mutex> lock(mtx);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return fail(TC_ERR_CUDA, "tc_pagerank_pull_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(addr[dev]);
    return TC_OK;
}

}  // namespace noalloc
}  // namespace tc

extern "C" int tc_pagerank_pull_noalloc(int32_t V, const int32_t *in_rowptr, const int32_t *in_colidx,
                                        const int32_t *out_degree, float damping, int32_t iters, int32_t dangling,
                                        float *ranks_out, void *stream) {
    using namespace tc;
    using namespace tc::noalloc;
    if (V < 1 || (int64_t)V > MAX_V)
        return fail(TC_ERR_UNSUPPORTED,
                    "tc_pagerank_pull_noalloc: V=%d outside [1, %lld] (the static scratch holds %lld vertices)", V,
                    (long long)MAX_V, (long long)MAX_V);
    if (!in_rowptr || !in_colidx || !out_degree || !ranks_out)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_pull_noalloc: null pointer");
    if (!(damping >= 0.0f && damping <= 1.0f) || iters < 0)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_pull_noalloc: damping outside [0,1] or iters < 0");
    if (dangling != TC_DANGLING_REDISTRIBUTE && dangling != TC_DANGLING_DROP)
        return fail(TC_ERR_INVALID_ARG, "tc_pagerank_pull_noalloc: bad dangling mode");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    TC_TRY(scratch_address(&base));
    const Layout l = layout(base);
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    int per_sm = 1;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gather, THREADS, 0));
    int64_t grid = (int64_t)caps.sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (((int64_t)V + 31) / 32 + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    if (grid > MAX_CTAS) grid = MAX_CTAS;
    if (grid < 1) grid = 1;
    // the array keeps the previous call's contents: re-arm the reduction counter
    TC_CUDA(cudaMemsetAsync(l.counter, 0, sizeof(unsigned), s));
    k_init<<<(unsigned)grid, THREADS, 0, s>>>(V, out_degree, l, iters == 0 ? ranks_out : nullptr);
    TC_LAUNCH_CHECK();
    const float base_term = (1.0f - damping) / (float)V;
    for (int it = 0; it < iters; ++it) {
        k_gather<<<(unsigned)grid, THREADS, 0, s>>>(in_rowptr, in_colidx, V, l, it & 1, base_term, damping,
                                                    dangling == TC_DANGLING_DROP, it == iters - 1 ? ranks_out : nullptr);
        TC_LAUNCH_CHECK();
    }
    return TC_OK;
}
