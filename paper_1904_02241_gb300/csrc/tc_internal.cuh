// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "tocab.h"

namespace tc {

// ---- error handling -------------------------------------------------------------------
void set_error(const char *fmt, ...);
int fail(int status, const char *fmt, ...);   // sets last error, returns status

#define TC_CUDA(call)                                                                   \
    do {                                                                                \
        cudaError_t err__ = (call);                                                     \
        if (err__ != cudaSuccess) {                                                     \
            return ::tc::fail(err__ == cudaErrorMemoryAllocation ? TC_ERR_OOM           \
                                                                 : TC_ERR_CUDA,         \
                              "%s failed at %s:%d: %s", #call, __FILE__, __LINE__,      \
                              cudaGetErrorString(err__));                               \
        }                                                                               \
    } while (0)

#define TC_LAUNCH_CHECK() TC_CUDA(cudaGetLastError())

#define TC_TRY(expr)                    \
    do {                                \
        int st__ = (expr);              \
        if (st__ != TC_OK) return st__; \
    } while (0)

// ---- division by a launch-invariant divisor ---------------------------------------------
// key / d for 0 <= key < 2^31 and d >= 1 as a multiply and a shift (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994): with l = ceil(log2 d),
// m = ceil(2^(31+l) / d) and s = 31 + l, (key * m) >> s = key / d exactly, because the error
// key * (m*d - 2^s) / (d * 2^s) stays below 2^-l <= 1/d; m <= 2^32 keeps key * m below 2^63.
struct DivBy {
    uint64_t m;
    int s;
};
inline DivBy div_by(int32_t d) {
    int l = 0;
    while (((int64_t)1 << l) < (int64_t)d) ++l;
    DivBy q;
    q.s = 31 + l;
    q.m = (((uint64_t)1 << q.s) + (uint64_t)d - 1) / (uint64_t)d;
    return q;
}
__device__ __forceinline__ int32_t div_apply(int32_t key, DivBy q) {
    return (int32_t)(((uint64_t)(uint32_t)key * q.m) >> q.s);
}

// ---- device block cache -----------------------------------------------------------------
// Preprocessing allocates and frees GB-sized temporaries on every call, and a fresh
// cudaMalloc/cudaFree of that size costs milliseconds (page mapping, plus the device-wide
// synchronisation inside cudaFree).  Freed blocks are therefore kept per device and handed
// out again for requests of between half and all of their size.  Returning a block
// synchronises the device first, exactly as cudaFree would, so no kernel still in flight can
// see its memory reused.  At most cache_limit bytes stay cached (larger leftovers go back to
// the driver), and an allocation that fails empties the cache and retries once.
cudaError_t cache_alloc(size_t n, void **p, size_t *got, int *device);
void cache_free(void *p, size_t bytes, int device);
size_t cache_limit();
size_t cache_held();                // bytes obtained from the driver and not returned
void cache_set_limit(size_t bytes);  // 0: no cap
size_t cache_get_limit();

// ---- device buffer that frees itself --------------------------------------------------
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    int device = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cache_free(p, bytes, device);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n) {  // grows only
        if (n <= bytes && p) return TC_OK;
        release();
        if (n == 0) n = 16;
        size_t got = 0;
        cudaError_t e = cache_alloc(n, &p, &got, &device);
        if (e != cudaSuccess) {
            p = nullptr;
            if (cache_get_limit())
                return fail(TC_ERR_OOM, "device allocation of %zu bytes refused: %s (memory cap %zu bytes, %zu held)",
                            n, cudaGetErrorString(e), cache_get_limit(), cache_held());
            return fail(TC_ERR_OOM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = got;
        return TC_OK;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void swap(DevBuf &o) {
        void *tp = p;
        p = o.p;
        o.p = tp;
        const size_t tb = bytes;
        bytes = o.bytes;
        o.bytes = tb;
        const int td = device;
        device = o.device;
        o.device = td;
    }
};

struct DeviceCaps {
    int device = 0;
    int sms = 0;
    int64_t l2_bytes = 0;
    int max_smem_optin = 0;
};
int device_caps(DeviceCaps *caps);

// ---- primitives (tc_prims.cu) -----------------------------------------------------------
// Exclusive scan of n int32 values into int64 out (out may not alias in); writes n outputs.
int scan_i32_to_i64(const int32_t *in, int64_t n, int64_t *out, cudaStream_t s);
int scan_i64(const int64_t *in, int64_t n, int64_t *out, cudaStream_t s);
int scan_i32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t s);  // total < 2^31
// The same scan with caller scratch (scan_ws_elems(n) int64 words): no allocation and no
// synchronisation, so it can sit between kernels of a level loop.
int64_t scan_ws_elems(int64_t n);
int scan_i32_to_i64_ws(const int32_t *in, int64_t n, int64_t *out, int64_t *ws, cudaStream_t s);
int head_tiles(const uint8_t *head, int64_t E, DevBuf *prefix, int64_t *R, cudaStream_t s);
int head_fill(const uint8_t *head, int64_t E, const int32_t *prefix, const int32_t *row, int32_t *rowptr,
              int32_t *id_map, cudaStream_t s);

// Stable sort of (key, val) int32 pairs by bucket(key) for bucket values < 2^bits,
// where bucket(key) = key / divisor (divisor >= 1).  LSD passes of 8 bits.
// Results land in (k_out, v_out); k_tmp/v_tmp are scratch of n elements each.
int stable_bucket_sort(const int32_t *k_in, const int32_t *v_in, int32_t *k_out, int32_t *v_out,
                       int32_t *k_tmp, int32_t *v_tmp, int64_t n, int32_t divisor, int bits,
                       cudaStream_t s);

// rowptr[v] = first i with keys[i] >= v, for v in [0, V]; keys sorted ascending, n keys.
int offsets_from_sorted(const int32_t *keys, int64_t n, int32_t V, int32_t *rowptr,
                        cudaStream_t s);
// Expand CSR rows into a per-edge row id array.
int expand_rows(const int32_t *rowptr, int32_t V, int32_t *row_of_edge, cudaStream_t s);

// ---- handles -------------------------------------------------------------------------------
struct Workspace;  // per-graph reusable scratch for the iteration drivers

}  // namespace tc

struct tc_graph {
    int32_t V = 0;
    int64_t E = 0;
    int device = 0;
    tc::DevBuf out_rowptr, out_colidx;  // G
    tc::DevBuf in_rowptr, in_colidx;    // G^T
    tc::DevBuf inv_outdeg;              // float[V], 0 for dangling vertices
    int32_t max_in_degree = 0, max_out_degree = 0;
    int64_t num_dangling = 0;
    // rows above the hub degree, for the unblocked kernels (CTA per row)
    int32_t hub_degree = 2048;
    int32_t num_in_hubs = 0, num_out_hubs = 0;
    tc::DevBuf in_hubs, out_hubs;
    // reusable scratch (grown on demand, freed with the graph)
    tc::DevBuf ws_contrib, ws_scalars, ws_partials, ws_bits, ws_misc;
    tc::DevBuf ws_queue, ws_qcnt, ws_qpos, ws_scan;  // BFS push levels
    tc::DevBuf ws_res;  // BFS resident push levels: range queues, counter slots, exit state, trace
    unsigned long long *h_counts = nullptr;  // pinned host words read after each BFS level (8 words)
    // source of every out-edge (edge-parallel push), built on first use
    bool push_esrc_built = false;
    tc::DevBuf push_esrc;
    // vertex numbering by out-degree and G^T in it, built on first use by the PPR batch
    bool ord_built = false;
    int32_t ord_ni = 0;
    tc::DevBuf ord_perm, ord_inv, ord_inv_outdeg, ord_rowptr, ord_colidx;
    // the PPR batch's persistent launch: its buffers (for one padded column count ppr_np), the
    // long rows' pieces, the autotuned hot block, and the captured launch with what it was built for
    int32_t ppr_np = 0, ppr_nhubs = 0, ppr_npieces = 0;
    int32_t ppr_hot = -1, ppr_tile = -1;  // evict-last source rows and tile width (-1: not tuned)
    tc::DevBuf ppr_C, ppr_D, ppr_src_old, ppr_src, ppr_isrc, ppr_sync, ppr_hub_rows, ppr_hub_p0, ppr_pieces, ppr_Ppc,
        ppr_hubcnt;
    // the rows without the in-edges of the long ones, and the runs of rows the queue hands out
    bool ppr_light_built = false;
    int32_t ppr_nchunks = 0;
    tc::DevBuf ppr_rowptr_l, ppr_colidx_l, ppr_islong, ppr_chunks;
    cudaGraphExec_t ppr_exec = nullptr;
    const void *ppr_key_out = nullptr;
    int32_t ppr_key_n = -1, ppr_key_iters = -1, ppr_key_hot = -1, ppr_key_grid = -1, ppr_key_tile = -1;
    float ppr_key_damping = -1.0f;
    ~tc_graph() {
        if (h_counts) cudaFreeHost(h_counts);
        if (ppr_exec) cudaGraphExecDestroy(ppr_exec);
    }
};

struct tc_part {
    const tc_graph *g = nullptr;
    int32_t dir = TC_PULL;
    int32_t B = 1, W = 1;
    int32_t V = 0;
    int64_t E = 0, R = 0;
    int32_t k = 1024;           // merge range width
    int32_t nranges = 0;        // ceil(V / k)
    int32_t hub_degree = 2048;
    int32_t num_hubs = 0;
    int64_t num_groups = 0;     // 32-row groups over the row space
    int64_t *h_blk_rows = nullptr, *h_blk_edges = nullptr;  // host copies [B+1]
    tc::DevBuf rowptr;          // int32[R+1] (global edge offsets)
    tc::DevBuf id_map;          // int32[R]
    tc::DevBuf colidx;          // int32[E]
    tc::DevBuf merge_off;       // int32[B * (nranges+1)]
    tc::DevBuf hubs;            // int32[num_hubs] rows with degree > hub_degree
    tc::DevBuf partial;         // float[R] partial sums (scratch)
    tc::DevBuf rowbits;         // uint32[ceil(R/32)] local next bits (BFS scratch)
    tc::DevBuf merge_offT;      // int32[(nranges+1) * B]: merge_off transposed (range-major)
    tc::DevBuf merge_gpre;      // int32[nranges * (B+1)]: per range, granules of MERGE_GRAN local
                                // rows before each block's slice (exclusive prefix; [B] = total)
    tc::DevBuf blk_rows_dev;    // int64[B+1]
    tc::DevBuf esrc;            // push only: int32[E] source (global) of every edge, for the
                                // edge-parallel scatter
    bool pperm_built = false, has_vals = false;  // push: values of the matrix (GC-pull SpMV)
    tc::DevBuf pperm;           // int32[E]: the loaded CSR position of every partition entry
    tc::DevBuf pvals;           // float[E]: the matrix values in partition order
    int32_t nptiles = 0;        // push, W * 8 bytes within shared memory: tiles of the staged push
    tc::DevBuf ptiles;          // int4[nptiles]: (block, first edge low 31 bits, high bits, edges)
    // ---- shared-memory staged format (pull, W <= smem capacity; see tc_tile.cu) ----
    bool tiled = false;
    int64_t padded_edges = 0;   // edges of the staged stream (blocks padded to TILE_WCHUNK)
    tc::DevBuf col16;           // uint16[padded_edges]: source - b*W
    tc::DevBuf heads;           // 1 bit per staged edge: a local row starts here
    tc::DevBuf id16;            // uint16[R]: id_map[r] minus the first vertex of its merge range
    tc::DevBuf lb_tab;          // int32[B]: per-block warp_min of the unstaged gathers (optional)
    int32_t ntiles = 0;         // CTAs of the staged gather: row-aligned tiles of equal estimated cost
    tc::DevBuf tile_blk;        // int32[ntiles]: block of every tile, in launch order (largest first)
    tc::DevBuf wtab;            // int2[ntiles * 33]: per tile and warp, (first staged edge, first row)
    // ---- vertex renumbering (TC_ORDER_OUTDEGREE); everything above is in the new numbering ----
    int32_t order = TC_ORDER_NATURAL;
    int32_t nz_out = 0;         // vertices with out-edges; renumbered: exactly the IDs below nz_out
    int32_t ni = 0;             // renumbered: the IDs from ni on have no edge at all (else ni = V)
    tc::DevBuf perm;            // int32[V]: original ID of new vertex n (renumbered only)
    tc::DevBuf inv_outdeg;      // float[V] in the new numbering (renumbered only)
    tc::DevBuf rstart;          // int32[nranges+1]: first vertex of every merge range (renumbered
                                // only; natural partitions use ranges [j*k, (j+1)*k))
    // ---- direct pieces (renumbered pull): single-edge pieces of the first Bd blocks ----
    int32_t Bd = 0;             // blocks whose single-edge pieces are direct
    int64_t ndirect = 0;
    tc::DevBuf dir_off;         // int32[nranges+1]: first direct piece of every merge range
    tc::DevBuf dir_u;           // int32[ndirect + 8]: source (new ID), sorted by target
    tc::DevBuf dir_id16;        // uint16[ndirect + 8]: target minus its range's first vertex
    ~tc_part() {
        delete[] h_blk_rows;
        delete[] h_blk_edges;
    }
};

namespace tc {
// The pull merge reads local rows in aligned granules of MERGE_GRAN entries (tc_pagerank.cu).
constexpr int MERGE_GRAN = 8;
// Shared-memory staged TOCAB format (tc_tile.cu).
constexpr int TILE_WCHUNK = 512;         // edges a warp streams per step (16 per lane)
constexpr int TILE_THREADS = 1024;
size_t tile_smem_bytes(int32_t W);       // dynamic shared memory of the staged gather for width W
int32_t tile_max_width(int max_smem_optin);
// Staged push (tc_push.cu): widest destination range in shared memory, its tiles, the scatter.
int32_t push_smem_width(int max_smem_optin);
int build_push_tiles(tc_part *p, int sms, cudaStream_t s);
int launch_push_smem(const tc_part *p, const float *contrib, void *sums, const double *fx_scale, bool fixed,
                     cudaStream_t s);
int build_tiles(tc_part *p, int sms, cudaStream_t s);
size_t merge_smem_bytes(int32_t k, int32_t B);   // dynamic shared memory of the ordered pull merge
size_t merge_atomic_smem_bytes(int32_t k, int32_t B, bool fixed);  // ... of the one-accumulator merges
// Launch the staged gather (+ long rows) writing p->partial from contributions `contrib`.
int launch_tiled_gather(const tc_part *p, const float *contrib, int *err_flag, cudaStream_t s, int *launches);

// The vertex numbering by out-degree (highest first, ties by ID, vertices without any edge last;
// tc_partition.cu): perm[n] = old ID of new vertex n, inv = its inverse, inv_outdeg in the new
// order, G^T renumbered (rp_new, ci_new; sources of a row in their old order), optionally the row
// of every edge of it (row may be null), and ni = the vertices with some edge.  Synchronises.
int order_by_outdegree(const tc_graph *g, cudaStream_t s, DevBuf *perm, DevBuf *inv, DevBuf *inv_outdeg,
                       DevBuf *rp_new, DevBuf *ci_new, DevBuf *row, int32_t *ni);

// L2 access-policy window over vertex values a kernel reads repeatedly (the block's values that
// Sec. 3.1 sizes to the last-level cache).  For one call, the context's persisting set-aside is
// raised to cover them (as far as the device allows), each launch carries a window that marks
// hits on them persisting and misses streaming, so streamed data cannot evict them; at the end
// the persisting lines are reset and the previous set-aside restored, after the stream has
// drained.
struct L2Window {
    bool on = false;
    size_t old_limit = 0, setaside = 0, max_window = 0;
    cudaStream_t s = nullptr;
    int begin(size_t want, cudaStream_t stream) {
        int dev = 0, max_persist = 0, max_win = 0;
        TC_CUDA(cudaGetDevice(&dev));
        TC_CUDA(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev));
        TC_CUDA(cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev));
        if (max_persist <= 0 || max_win <= 0) return TC_OK;  // no set-aside: the call runs without
        TC_CUDA(cudaDeviceGetLimit(&old_limit, cudaLimitPersistingL2CacheSize));
        setaside = want < (size_t)max_persist ? want : (size_t)max_persist;
        max_window = (size_t)max_win;
        s = stream;
        TC_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, setaside));
        on = true;
        return TC_OK;
    }
    cudaAccessPolicyWindow window(const void *base, size_t bytes) const {
        cudaAccessPolicyWindow w = {};
        w.base_ptr = const_cast<void *>(base);
        w.num_bytes = bytes < max_window ? bytes : max_window;
        w.hitRatio = w.num_bytes > setaside ? (float)((double)setaside / (double)w.num_bytes) : 1.0f;
        w.hitProp = cudaAccessPropertyPersisting;
        w.missProp = cudaAccessPropertyStreaming;
        return w;
    }
    int end() {
        if (!on) return TC_OK;
        on = false;
        cudaError_t e = cudaStreamSynchronize(s);
        cudaError_t e2 = cudaCtxResetPersistingL2Cache();
        cudaError_t e3 = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, old_limit);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = e3;
        if (e != cudaSuccess) return fail(TC_ERR_CUDA, "L2 window: %s", cudaGetErrorString(e));
        return TC_OK;
    }
    ~L2Window() { end(); }
};

// Rows of a CSR with more than `min_degree` edges, as a compact int32 list (ascending).
int collect_hubs(const int32_t *rowptr, int64_t nrows, int32_t min_degree, DevBuf *list, int32_t *count,
                 cudaStream_t s);
}  // namespace tc
