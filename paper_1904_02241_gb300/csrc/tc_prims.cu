// Error reporting, device capabilities and the device primitives used by preprocessing:
// exclusive scans, a stable LSD bucket sort, offsets from sorted keys, row expansion.
#include <stdarg.h>

#include <map>
#include <mutex>

#include "tc_internal.cuh"

namespace tc {

// ---- device block cache -----------------------------------------------------------------
namespace {
struct CachedBlock {
    void *p;
    uint64_t seq;  // when it was freed: the cache evicts the least recently freed first
};
struct BlockCache {
    std::mutex mu;
    std::multimap<std::pair<int, size_t>, CachedBlock> free_blocks;  // (device, bytes) -> block
    uint64_t next_seq = 0;
    size_t cached = 0;
    size_t held = 0;   // bytes obtained from cudaMalloc and not yet returned to the driver
    size_t limit = 0;  // 0: no cap
    void drop_all() {  // caller holds mu
        int cur = -1;
        cudaGetDevice(&cur);
        for (auto &kv : free_blocks) {
            cudaSetDevice(kv.first.first);
            cudaFree(kv.second.p);
            held -= kv.first.second;
        }
        if (cur >= 0) cudaSetDevice(cur);
        free_blocks.clear();
        cached = 0;
    }
};
BlockCache &block_cache() {
    static BlockCache *c = new BlockCache();  // never destroyed: frees at exit would race the driver teardown
    return *c;
}
}  // namespace

size_t cache_limit() { return size_t(16) << 30; }

cudaError_t cache_alloc(size_t n, void **p, size_t *got, int *device) {
    n = (n + 255) & ~size_t(255);
    cudaError_t e = cudaGetDevice(device);
    if (e != cudaSuccess) return e;
    BlockCache &c = block_cache();
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto it = c.free_blocks.lower_bound({*device, n});
        if (it != c.free_blocks.end() && it->first.first == *device && it->first.second <= 2 * n) {
            *p = it->second.p;
            *got = it->first.second;
            c.cached -= *got;
            c.free_blocks.erase(it);
            return cudaSuccess;
        }
    }
    {  // the caller's memory cap: cached blocks are released first, then the request is refused
        std::lock_guard<std::mutex> lk(c.mu);
        if (c.limit && c.held + n > c.limit) c.drop_all();
        if (c.limit && c.held + n > c.limit) return cudaErrorMemoryAllocation;
    }
    e = cudaMalloc(p, n);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        {
            std::lock_guard<std::mutex> lk(c.mu);
            c.drop_all();
        }
        e = cudaMalloc(p, n);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e;
    }
    *got = n;
    std::lock_guard<std::mutex> lk(c.mu);
    c.held += n;
    return cudaSuccess;
}

size_t cache_held() {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return c.held;
}

void cache_set_limit(size_t bytes) {
    cudaDeviceSynchronize();  // cached blocks may go back to the driver below
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.limit = bytes;
    if (bytes) c.drop_all();  // a cap counts what is held: release the cached blocks first
}

size_t cache_get_limit() {
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return c.limit;
}

void cache_free(void *p, size_t bytes, int device) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    cudaDeviceSynchronize();  // the same ordering guarantee cudaFree gives
    BlockCache &c = block_cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (bytes > cache_limit()) {
        cudaFree(p);
        c.held -= bytes;
    } else {
        c.free_blocks.insert({{device, bytes}, CachedBlock{p, c.next_seq++}});
        c.cached += bytes;
        // evict the least recently freed blocks until the cache fits its limit again: a job that
        // runs again asks for the sizes it freed last (evicting the largest first dropped
        // exactly those, the big temporaries of graph load and partition)
        while (c.cached > cache_limit() && !c.free_blocks.empty()) {
            auto old = c.free_blocks.begin();
            for (auto it = c.free_blocks.begin(); it != c.free_blocks.end(); ++it)
                if (it->second.seq < old->second.seq) old = it;
            cudaSetDevice(old->first.first);
            cudaFree(old->second.p);
            c.cached -= old->first.second;
            c.held -= old->first.second;
            c.free_blocks.erase(old);
        }
    }
    if (cur >= 0) cudaSetDevice(cur);
}

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

// A thread's SCAN_ITEMS consecutive inputs (8 items start 32- or 64-byte aligned: vector
// loads for whole groups, element loads at the ragged end).
template <class Tin, class Tout>
__device__ __forceinline__ void load_items(const Tin *in, int64_t n, int64_t base, bool vec, Tout (&v)[SCAN_ITEMS]) {
    static_assert(SCAN_ITEMS == 8, "vector loads assume 8 items");
    if (vec && base + SCAN_ITEMS <= n) {
        if (sizeof(Tin) == 1) {
            const uint2 w = *reinterpret_cast<const uint2 *>(in + base);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i] = (Tout)((w.x >> (8 * i)) & 0xFFu);
                v[4 + i] = (Tout)((w.y >> (8 * i)) & 0xFFu);
            }
        } else if (sizeof(Tin) == 4) {
            const int4 *p = reinterpret_cast<const int4 *>(in + base);
            const int4 a = p[0], b = p[1];
            const int32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = (Tout)w[i];
        } else {
            const longlong2 *p = reinterpret_cast<const longlong2 *>(in + base);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const longlong2 x = p[i];
                v[2 * i] = (Tout)x.x;
                v[2 * i + 1] = (Tout)x.y;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) v[i] = (base + i < n) ? (Tout)in[base + i] : Tout(0);
    }
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const Tin *in, int64_t n, Tout *tile_sums, bool vec) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    load_items(in, n, base, vec, v);
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) s += v[i];
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
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const Tin *in, int64_t n, const Tout *tile_prefix, Tout *out, bool vec) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    load_items(in, n, base, vec, v);
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) s += v[i];
    __shared__ Tout total;
    Tout run = block_exclusive_sum<Tout>(s, &total);
    run += tile_prefix ? tile_prefix[blockIdx.x] : Tout(0);
    Tout o[SCAN_ITEMS];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        o[i] = run;
        run += v[i];
    }
    if (vec && base + SCAN_ITEMS <= n) {  // 8 aligned items per thread: 16-byte stores
        if (sizeof(Tout) == 8) {
            longlong2 *q = reinterpret_cast<longlong2 *>(out + base);
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS / 2; ++i) q[i] = make_longlong2((long long)o[2 * i], (long long)o[2 * i + 1]);
        } else {
            int4 *q = reinterpret_cast<int4 *>(out + base);
#pragma unroll
            for (int i = 0; i < SCAN_ITEMS / 4; ++i)
                q[i] = make_int4((int)o[4 * i], (int)o[4 * i + 1], (int)o[4 * i + 2], (int)o[4 * i + 3]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (base + i < n) out[base + i] = o[i];
    }
}

template <class Tin, class Tout>
static int scan_impl(const Tin *in, int64_t n, Tout *out, cudaStream_t s) {
    if (n <= 0) return TC_OK;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    // vector access needs 8 items' worth of alignment on both sides
    const bool vec = ((uintptr_t)in % (8 * sizeof(Tin))) == 0 && ((uintptr_t)out % (8 * sizeof(Tout))) == 0;
    if (tiles == 1) {
        k_scan_apply<Tin, Tout><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out, vec);
        TC_LAUNCH_CHECK();
        return TC_OK;
    }
    DevBuf sums, pref;
    TC_TRY(sums.alloc(tiles * sizeof(Tout)));
    TC_TRY(pref.alloc(tiles * sizeof(Tout)));
    k_scan_reduce<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums.as<Tout>(), vec);
    TC_LAUNCH_CHECK();
    TC_TRY((scan_impl<Tout, Tout>(sums.as<Tout>(), tiles, pref.as<Tout>(), s)));
    k_scan_apply<Tin, Tout><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, pref.as<Tout>(), out, vec);
    TC_LAUNCH_CHECK();
    // DevBuf frees are stream-unordered: make sure the kernels using them are done.
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

// ---- row starts of a sorted edge list ---------------------------------------------------
// head[i] = 1 where edge i starts a row.  head_tiles: exclusive prefix of the head counts per
// scan tile (prefix[t]) and their total R.  head_fill: for every head i with rank r among the
// heads, rowptr[r] = i and id_map[r] = row[i] (a scan whose result is written only at heads,
// so no per-edge row number array is stored).
__global__ void __launch_bounds__(SCAN_THREADS) k_head_fill(const uint8_t *head, int64_t n, const int32_t *tile_prefix,
                                                           const int32_t *row, int32_t *rowptr, int32_t *id_map) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    load_items(head, n, base, true, v);
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) s += v[i];
    __shared__ int32_t total;
    int32_t run = block_exclusive_sum<int32_t>(s, &total) + tile_prefix[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (v[i]) {
            rowptr[run] = (int32_t)(base + i);
            id_map[run] = row[base + i];
            ++run;
        }
    }
}

int head_tiles(const uint8_t *head, int64_t E, DevBuf *prefix, int64_t *R, cudaStream_t s) {
    *R = 0;
    if (E <= 0) return TC_OK;
    if ((uintptr_t)head % 8 != 0) return fail(TC_ERR_INVALID_ARG, "head_tiles: head must be 8-byte aligned");
    const int64_t tiles = (E + SCAN_TILE - 1) / SCAN_TILE;
    DevBuf sums;
    TC_TRY(sums.alloc((size_t)tiles * 4));
    TC_TRY(prefix->alloc((size_t)tiles * 4));
    k_scan_reduce<uint8_t, int32_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(head, E, sums.as<int32_t>(), true);
    TC_LAUNCH_CHECK();
    TC_TRY((scan_impl<int32_t, int32_t>(sums.as<int32_t>(), tiles, prefix->as<int32_t>(), s)));
    int32_t last[2] = {0, 0};
    TC_CUDA(cudaMemcpyAsync(&last[0], prefix->as<int32_t>() + tiles - 1, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(&last[1], sums.as<int32_t>() + tiles - 1, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    *R = (int64_t)last[0] + last[1];
    return TC_OK;
}

int head_fill(const uint8_t *head, int64_t E, const int32_t *prefix, const int32_t *row, int32_t *rowptr,
              int32_t *id_map, cudaStream_t s) {
    if (E <= 0) return TC_OK;
    const int64_t tiles = (E + SCAN_TILE - 1) / SCAN_TILE;
    k_head_fill<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(head, E, prefix, row, rowptr, id_map);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

int64_t scan_ws_elems(int64_t n) {
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    return tiles <= 1 ? 0 : 2 * tiles + scan_ws_elems(tiles);
}

template <class Tin>
static int scan_ws_impl(const Tin *in, int64_t n, int64_t *out, int64_t *ws, cudaStream_t s) {
    if (n <= 0) return TC_OK;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    const bool vec = ((uintptr_t)in % (8 * sizeof(Tin))) == 0 && ((uintptr_t)out % 64) == 0;
    if (tiles == 1) {
        k_scan_apply<Tin, int64_t><<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out, vec);
        TC_LAUNCH_CHECK();
        return TC_OK;
    }
    int64_t *sums = ws, *pref = ws + tiles;
    k_scan_reduce<Tin, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums, vec);
    TC_LAUNCH_CHECK();
    TC_TRY(scan_ws_impl<int64_t>(sums, tiles, pref, ws + 2 * tiles, s));
    k_scan_apply<Tin, int64_t><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, pref, out, vec);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

int scan_i32_to_i64_ws(const int32_t *in, int64_t n, int64_t *out, int64_t *ws, cudaStream_t s) {
    return scan_ws_impl<int32_t>(in, n, out, ws, s);
}

int scan_i32_to_i64(const int32_t *in, int64_t n, int64_t *out, cudaStream_t s) {
    return scan_impl<int32_t, int64_t>(in, n, out, s);
}
int scan_i32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t s) { return scan_impl<int32_t, int32_t>(in, n, out, s); }
int scan_i64(const int64_t *in, int64_t n, int64_t *out, cudaStream_t s) { return scan_impl<int64_t, int64_t>(in, n, out, s); }

// ----------------------------------------------------------------------------------------
// Stable LSD bucket sort: 8-bit digits of key/divisor (256 buckets; one 9-bit pass with 512
// buckets for 9-bit keys), tiles of 4096 items.
// Each pass is a per-tile histogram, an exclusive scan of the bucket-major count table and a
// stable scatter; stability is what keeps in-rows sorted by source.
// ----------------------------------------------------------------------------------------
constexpr int RX_THREADS = 256;
constexpr int RX_ROUNDS = 16;
constexpr int RX_TILE = RX_THREADS * RX_ROUNDS;
constexpr int RX_BUCKETS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;

// Digit of key / divisor: the multiply-and-shift of DivBy with the digit's shift folded into
// the same shift.
struct RxDigit {
    uint64_t m;
    int sh;
};
static RxDigit rx_digit(int32_t divisor, int shift) {
    const DivBy q = div_by(divisor);
    RxDigit r;
    r.m = q.m;
    r.sh = q.s + shift;
    if (r.sh > 63) {  // key * m < 2^63: this digit is zero for every key
        r.m = 0;
        r.sh = 0;
    }
    return r;
}
template <int NB>
__device__ __forceinline__ int rx_bucket(int32_t key, RxDigit dg) {
    return (int)(((uint64_t)(uint32_t)key * dg.m) >> dg.sh) & (NB - 1);
}

// Per-tile bucket counts (NB = 256 or 512 buckets).  All 16 keys of a thread are loaded before
// any counting so that the loads overlap; every warp counts into its own shared histogram
// (plain shared atomics: keys of one warp rarely share a bucket), and the 8 warp histograms
// are summed at the end.
template <int NB>
__global__ void __launch_bounds__(RX_THREADS) k_rx_hist(const int32_t *keys, int64_t n, RxDigit dg,
                                                        int32_t *counts, int64_t ntiles) {
    __shared__ int32_t h[RX_WARPS][NB];
    const int warp = threadIdx.x >> 5;
    for (int w = 0; w < RX_WARPS; ++w)
        for (int b = threadIdx.x; b < NB; b += RX_THREADS) h[w][b] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RX_TILE;
    int32_t k[RX_ROUNDS];
#pragma unroll
    for (int r = 0; r < RX_ROUNDS; ++r) {
        const int64_t i = base + r * RX_THREADS + threadIdx.x;
        k[r] = (i < n) ? keys[i] : -1;
    }
#pragma unroll
    for (int r = 0; r < RX_ROUNDS; ++r) {
        const int64_t i = base + r * RX_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&h[warp][rx_bucket<NB>(k[r], dg)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < NB; b += RX_THREADS) {
        int tot = 0;
        for (int w = 0; w < RX_WARPS; ++w) tot += h[w][b];
        counts[(int64_t)b * ntiles + blockIdx.x] = tot;
    }
}

// Stable scatter of one tile.  Warp w owns items [w*512, (w+1)*512) of the tile, 16 rounds of
// 32 in order, held in registers.  (A) count per warp and bucket with match masks, noting each
// item's rank among the warp's items of its bucket;  (B) each thread takes NB/256 consecutive
// buckets and turns their counts into per-warp offsets inside the tile's bucket-ordered layout
// (warps in order, buckets by a CTA scan);  (C) every item goes to its slot in shared memory;
// (D) consecutive threads copy consecutive slots out, so each bucket run of the tile leaves as
// one contiguous store stream.  Equal buckets keep their input order throughout.
constexpr int RX_PER_WARP = RX_TILE / RX_WARPS;  // 512
constexpr int RX_WROUNDS = RX_PER_WARP / 32;     // 16
template <int NB>
constexpr size_t rx_scatter_smem() {
    return (size_t)RX_TILE * 8 + (size_t)RX_WARPS * NB * 4 + (size_t)NB * 4 + (size_t)NB * 8;
}
template <int NB>
__global__ void __launch_bounds__(RX_THREADS) k_rx_scatter(const int32_t *kin, const int32_t *vin, int32_t *kout,
                                                           int32_t *vout, int64_t n, RxDigit dg,
                                                           const int64_t *offs, int64_t ntiles) {
    constexpr int PER = NB / RX_THREADS;  // buckets per thread in (B)
    extern __shared__ __align__(16) unsigned char rsm[];
    int64_t *gdelta = reinterpret_cast<int64_t *>(rsm);                   // [NB] global run start minus lstart
    int32_t *skey = reinterpret_cast<int32_t *>(gdelta + NB);             // [RX_TILE]
    int32_t *sval = skey + RX_TILE;                                       // [RX_TILE]
    int32_t *wpos = sval + RX_TILE;                                       // [RX_WARPS][NB]
    int32_t *lstart = wpos + RX_WARPS * NB;                               // [NB]
    __shared__ int32_t wsum[RX_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int b = lane; b < NB; b += 32) wpos[warp * NB + b] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * RX_TILE;
    const int64_t base = tile0 + (int64_t)warp * RX_PER_WARP;
    int32_t key[RX_WROUNDS], val[RX_WROUNDS];
    uint32_t local[RX_WROUNDS / 2];  // rank of each item among its warp's items of its bucket (16 bits each)
#pragma unroll
    for (int r = 0; r < RX_WROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        key[r] = (i < n) ? kin[i] : 0;
        val[r] = (i < n) ? vin[i] : 0;
    }
    // (A) counts per warp and bucket, and each item's rank among them (earlier rounds first,
    // then lower lanes)
#pragma unroll
    for (int r = 0; r < RX_WROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        const int b = (i < n) ? rx_bucket<NB>(key[r], dg) : NB;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int prev = b < NB ? wpos[warp * NB + b] : 0;
        const uint32_t rank = (uint32_t)(prev + __popc(peers & lt_mask));
        if (r & 1) local[r >> 1] |= rank << 16;
        else local[r >> 1] = rank;
        __syncwarp();
        if (b < NB && (peers & lt_mask) == 0) wpos[warp * NB + b] = prev + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // (B) per-warp offsets inside each bucket, then a CTA scan of the bucket totals
    {
        int tot[PER];
        int run_all = 0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = threadIdx.x * PER + q;
            int run = 0;
            for (int w = 0; w < RX_WARPS; ++w) {
                const int c = wpos[w * NB + b];
                wpos[w * NB + b] = run;
                run += c;
            }
            tot[q] = run;
            run_all += run;
        }
        int inc = run_all;  // inclusive warp scan of the threads' totals
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        int ls = inc - run_all;
        for (int w = 0; w < warp; ++w) ls += wsum[w];
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const int b = threadIdx.x * PER + q;
            lstart[b] = ls;
            gdelta[b] = offs[(int64_t)b * ntiles + blockIdx.x] - ls;
            ls += tot[q];
        }
    }
    __syncthreads();
    // (C) every item to its slot of the tile's bucket-ordered layout
#pragma unroll
    for (int r = 0; r < RX_WROUNDS; ++r) {
        const int64_t i = base + r * 32 + lane;
        if (i < n) {
            const int b = rx_bucket<NB>(key[r], dg);
            const int slot = lstart[b] + wpos[warp * NB + b] + (int)((local[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
            skey[slot] = key[r];
            sval[slot] = val[r];
        }
    }
    __syncthreads();
    // (D)
    const int count = (int)((n - tile0) < RX_TILE ? (n - tile0) : RX_TILE);
    if (count == RX_TILE) {  // full tile: unrolled, so that the shared loads of several rounds overlap
#pragma unroll 8
        for (int q = 0; q < RX_ROUNDS; ++q) {
            const int t = q * RX_THREADS + threadIdx.x;
            const int32_t k = skey[t];
            const int64_t pos = gdelta[rx_bucket<NB>(k, dg)] + t;
            kout[pos] = k;
            vout[pos] = sval[t];
        }
    } else {
        for (int t = threadIdx.x; t < count; t += RX_THREADS) {
            const int32_t k = skey[t];
            const int64_t pos = gdelta[rx_bucket<NB>(k, dg)] + t;
            kout[pos] = k;
            vout[pos] = sval[t];
        }
    }
}

// One pass of the sort: digit of key / divisor at bit `shift`, NB buckets.
template <int NB>
static int rx_pass(const int32_t *ksrc, const int32_t *vsrc, int32_t *kd, int32_t *vd, int64_t n, int64_t ntiles,
                   int32_t divisor, int shift, DevBuf *counts, DevBuf *offs, cudaStream_t s) {
    TC_TRY(counts->alloc((size_t)ntiles * NB * sizeof(int32_t)));
    TC_TRY(offs->alloc((size_t)ntiles * NB * sizeof(int64_t)));
    const RxDigit dg = rx_digit(divisor, shift);
    k_rx_hist<NB><<<(unsigned)ntiles, RX_THREADS, 0, s>>>(ksrc, n, dg, counts->as<int32_t>(), ntiles);
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32_to_i64(counts->as<int32_t>(), ntiles * NB, offs->as<int64_t>(), s));
    constexpr size_t smem = rx_scatter_smem<NB>();
    TC_CUDA(cudaFuncSetAttribute(k_rx_scatter<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rx_scatter<NB><<<(unsigned)ntiles, RX_THREADS, smem, s>>>(ksrc, vsrc, kd, vd, n, dg, offs->as<int64_t>(),
                                                               ntiles);
    TC_LAUNCH_CHECK();
    return TC_OK;
}

int stable_bucket_sort(const int32_t *k_in, const int32_t *v_in, int32_t *k_out, int32_t *v_out,
                       int32_t *k_tmp, int32_t *v_tmp, int64_t n, int32_t divisor, int bits,
                       cudaStream_t s) {
    if (n <= 0) return TC_OK;
    if (divisor < 1) return fail(TC_ERR_INVALID_ARG, "stable_bucket_sort: divisor < 1");
    // 8-bit digits; a 9-bit key (up to 512 blocks) takes one 9-bit pass instead of two
    const bool nine = bits == 9;
    const int passes = nine ? 1 : (bits <= 0 ? 1 : (bits + 7) / 8);
    const int64_t ntiles = (n + RX_TILE - 1) / RX_TILE;
    DevBuf counts, offs;
    // ping-pong so that the last pass writes (k_out, v_out)
    const int32_t *ksrc = k_in, *vsrc = v_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        int32_t *kd = to_out ? k_out : k_tmp;
        int32_t *vd = to_out ? v_out : v_tmp;
        if (nine)
            TC_TRY(rx_pass<2 * RX_BUCKETS>(ksrc, vsrc, kd, vd, n, ntiles, divisor, 0, &counts, &offs, s));
        else
            TC_TRY(rx_pass<RX_BUCKETS>(ksrc, vsrc, kd, vd, n, ntiles, divisor, 8 * p, &counts, &offs, s));
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
// A warp takes 32 rows at a time: one coalesced load of their offsets, then the rows' edge
// ranges are filled one row after the other (no dependent load per row).
__global__ void k_expand_rows(const int32_t *rowptr, int32_t V, int32_t *row_of_edge) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; u0 < V; u0 += warps * 32) {
        const int64_t u = u0 + lane;
        int32_t b = 0, e = 0;
        if (u < V) {
            b = rowptr[u];
            e = rowptr[u + 1];
        }
        const int nrows = (V - u0) < 32 ? (int)(V - u0) : 32;
        for (int j = 0; j < nrows; ++j) {
            const int32_t bj = __shfl_sync(0xffffffffu, b, j), ej = __shfl_sync(0xffffffffu, e, j);
            for (int32_t i = bj + lane; i < ej; i += 32) row_of_edge[i] = (int32_t)(u0 + j);
        }
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

extern "C" int tc_set_device_memory_limit(int64_t bytes) {
    if (bytes < 0) return tc::fail(TC_ERR_INVALID_ARG, "tc_set_device_memory_limit: negative byte count");
    tc::cache_set_limit((size_t)bytes);
    return TC_OK;
}

extern "C" int64_t tc_device_memory_held(void) { return (int64_t)tc::cache_held(); }

extern "C" int tc_version(void) { return 100; }
