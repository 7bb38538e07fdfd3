// Error reporting, device capabilities and the device primitives used by preprocessing:
// exclusive scans, a stable LSD bucket sort, offsets from sorted keys, row expansion.
#include <stdarg.h>

#include "tc_internal.cuh"

namespace tc {

static thread_local char g_last_error[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

int fail(int status, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return status;
}

int device_caps(DeviceCaps *caps) {
    TC_CUDA(cudaGetDevice(&caps->device));
    int v = 0;
    TC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, caps->device));
    caps->sms = v;
    TC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, caps->device));
    caps->l2_bytes = v;
    TC_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, caps->device));
    caps->max_smem_optin = v;
    return TC_OK;
}

// ----------------------------------------------------------------------------------------
// Exclusive scan: tiles of 2048 elements (256 threads x 8 consecutive items).
// ----------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T block_exclusive_sum(T x, T *total) {
    __shared__ T warp_tot[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < SCAN_THREADS / 32 ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == SCAN_THREADS / 32 - 1) *total = wi;
    }
    __syncthreads();
    T r = warp_tot[warp] + incl - x;
    __syncthreads();
    return r;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const Tin *in, int64_t n, Tout *tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < n) s += (Tout)in[base + i];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    __shared__ Tout ws[SCAN_THREADS / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        Tout t = 0;
        for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
        tile_sums[blockIdx.x] = t;
    }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const Tin *in, int64_t n, const Tout *tile_prefix, Tout *out) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? (Tout)in[base + i] : Tout(0);
        s += v[i];
    }
    __shared__ Tout total;
    Tout run = block_exclusive_sum<Tout>(s, &total);
    run += tile_prefix ? tile_prefix[blockIdx.x] : Tout(0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
}

template <class Tin>
static int scan_impl(const Tin *in, int64_t n, int64_t *out, cudaStream_t s) {
    if (n <= 0) return TC_OK;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_scan_apply<Tin, int64_t><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out);
        TC_LAUNCH_CHECK();
        return TC_OK;
    }
    DevBuf sums, pref;
    TC_TRY(sums.alloc(tiles * sizeof(int64_t)));
    TC_TRY(pref.alloc(tiles * sizeof(int64_t)));
    k_scan_reduce<Tin, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums.as<int64_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_impl<int64_t>(sums.as<int64_t>(), tiles, pref.as<int64_t>(), s));
    k_scan_apply<Tin, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, pref.as<int64_t>(), out);
    TC_LAUNCH_CHECK();
    // DevBuf frees are stream-unordered: make sure the kernels using them are done.
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

int scan_i32_to_i64(const int32_t *in, int64_t n, int64_t *out, cudaStream_t s) { return scan_impl<int32_t>(in, n, out, s); }
int scan_i64(const int64_t *in, int64_t n, int64_t *out, cudaStream_t s) { return scan_impl<int64_t>(in, n, out, s); }

// ----------------------------------------------------------------------------------------
// Stable bucket pass: 256 buckets, tiles of 4096 items processed in 16 ordered rounds of
// 256 items; ranks inside a round come from warp match masks, so equal buckets keep their
// input order (stability is what keeps in-rows sorted by source).
// ----------------------------------------------------------------------------------------
constexpr int RX_THREADS = 256;
constexpr int RX_ROUNDS = 16;
constexpr int RX_TILE = RX_THREADS * RX_ROUNDS;
constexpr int RX_BUCKETS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;

__device__ __forceinline__ int rx_bucket(int32_t key, int32_t divisor, int shift) {
    return (int)(((uint32_t)key / (uint32_t)divisor) >> shift) & (RX_BUCKETS - 1);
}

__global__ void __launch_bounds__(RX_THREADS) k_rx_hist(const int32_t *keys, int64_t n, int32_t divisor, int shift,
                                                        int32_t *counts, int64_t ntiles) {
    __shared__ int32_t h[RX_BUCKETS];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RX_TILE;
    for (int r = 0; r < RX_ROUNDS; ++r) {
        int64_t i = base + r * RX_THREADS + threadIdx.x;
        const int b = (i < n) ? rx_bucket(keys[i], divisor, shift) : RX_BUCKETS;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        if (b < RX_BUCKETS && (peers & ((1u << (threadIdx.x & 31)) - 1u)) == 0)
            atomicAdd(&h[b], __popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RX_THREADS) k_rx_scatter(const int32_t *kin, const int32_t *vin, int32_t *kout,
                                                           int32_t *vout, int64_t n, int32_t divisor, int shift,
                                                           const int64_t *offs, int64_t ntiles) {
    __shared__ int64_t running[RX_BUCKETS];
    __shared__ int32_t wcnt[RX_WARPS][RX_BUCKETS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RX_TILE;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < RX_ROUNDS; ++r) {
        for (int w = 0; w < RX_WARPS; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t i = base + r * RX_THREADS + threadIdx.x;
        const bool valid = i < n;
        int32_t key = 0, val = 0;
        int b = RX_BUCKETS;  // sentinel for invalid lanes
        if (valid) {
            key = kin[i];
            val = vin[i];
            b = rx_bucket(key, divisor, shift);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) wcnt[warp][b] = __popc(peers);
        __syncthreads();
        if (valid) {
            int64_t pos = running[b] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][b];
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        int32_t add = 0;
        for (int w = 0; w < RX_WARPS; ++w) add += wcnt[w][threadIdx.x];
        running[threadIdx.x] += add;
        __syncthreads();
    }
}

int stable_bucket_sort(const int32_t *k_in, const int32_t *v_in, int32_t *k_out, int32_t *v_out,
                       int32_t *k_tmp, int32_t *v_tmp, int64_t n, int32_t divisor, int bits,
                       cudaStream_t s) {
    if (n <= 0) return TC_OK;
    if (divisor < 1) return fail(TC_ERR_INVALID_ARG, "stable_bucket_sort: divisor < 1");
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    const int64_t ntiles = (n + RX_TILE - 1) / RX_TILE;
    DevBuf counts, offs;
    TC_TRY(counts.alloc(ntiles * RX_BUCKETS * sizeof(int32_t)));
    TC_TRY(offs.alloc(ntiles * RX_BUCKETS * sizeof(int64_t)));
    // ping-pong so that the last pass writes (k_out, v_out)
    const int32_t *ksrc = k_in, *vsrc = v_in;
    for (int p = 0; p < passes; ++p) {
        const bool last = (p == passes - 1);
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        int32_t *kd = to_out ? k_out : k_tmp;
        int32_t *vd = to_out ? v_out : v_tmp;
        (void)last;
        k_rx_hist<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(ksrc, n, divisor, 8 * p, counts.as<int32_t>(), ntiles);
        TC_LAUNCH_CHECK();
        TC_TRY(scan_i32_to_i64(counts.as<int32_t>(), ntiles * RX_BUCKETS, offs.as<int64_t>(), s));
        k_rx_scatter<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(ksrc, vsrc, kd, vd, n, divisor, 8 * p,
                                                           offs.as<int64_t>(), ntiles);
        TC_LAUNCH_CHECK();
        ksrc = kd;
        vsrc = vd;
    }
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

// ----------------------------------------------------------------------------------------
__global__ void k_offsets_from_sorted(const int32_t *keys, int64_t n, int32_t V, int32_t *rowptr) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= V; v += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;  // first index with keys[i] >= v
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < v) lo = mid + 1; else hi = mid;
        }
        rowptr[v] = (int32_t)lo;
    }
}

int offsets_from_sorted(const int32_t *keys, int64_t n, int32_t V, int32_t *rowptr, cudaStream_t s) {
    DeviceCaps c;
    TC_TRY(device_caps(&c));
    k_offsets_from_sorted<<<c.sms * 8, 256, 0, s>>>(keys, n, V, rowptr);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

// One warp per row: lanes write the row id over the row's edge range.
__global__ void k_expand_rows(const int32_t *rowptr, int32_t V, int32_t *row_of_edge) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; u < V; u += warps) {
        const int32_t b = rowptr[u], e = rowptr[u + 1];
        for (int32_t i = b + lane; i < e; i += 32) row_of_edge[i] = (int32_t)u;
    }
}

int expand_rows(const int32_t *rowptr, int32_t V, int32_t *row_of_edge, cudaStream_t s) {
    if (V <= 0) return TC_OK;
    DeviceCaps c;
    TC_TRY(device_caps(&c));
    k_expand_rows<<<c.sms * 8, 256, 0, s>>>(rowptr, V, row_of_edge);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

}  // namespace tc

// ---- C ABI: status ---------------------------------------------------------------------------
extern "C" const char *tc_status_string(int status) {
    switch (status) {
        case TC_OK: return "TC_OK";
        case TC_ERR_INVALID_ARG: return "TC_ERR_INVALID_ARG";
        case TC_ERR_INVALID_GRAPH: return "TC_ERR_INVALID_GRAPH";
        case TC_ERR_OOM: return "TC_ERR_OOM";
        case TC_ERR_CUDA: return "TC_ERR_CUDA";
        case TC_ERR_TIMEOUT: return "TC_ERR_TIMEOUT";
        case TC_ERR_UNSUPPORTED: return "TC_ERR_UNSUPPORTED";
        default: return "TC_ERR_UNKNOWN";
    }
}

extern "C" const char *tc_last_error(void) { return tc::g_last_error; }

extern "C" int tc_version(void) { return 100; }
