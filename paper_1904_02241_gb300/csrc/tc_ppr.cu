// Personalised PageRank for a batch of sources (one column per source), pull direction.
// Column j follows Alg. 1 with the teleport term (1-d) and the dangling mass of column j sent
// to its own source s_j, starting from e_{s_j}:
//   R'[v,j] = d * sum_{u->v} R[u,j] / out_degree[u] + [v == s_j] ((1-d) + d * D_j),
//   D_j     = sum over dangling u of R[u,j].
// The batch is an FP32 [V x n] row-major matrix; one warp gathers whole rows of the
// contribution matrix (n floats, float4 per lane), so every in-edge costs one coalesced row
// read.  Per-column dangling sums are accumulated in 64-bit fixed point (deterministic).
#include "tc_common_dev.cuh"

namespace tc {

// Compensated (Kahan) addition of y into (sum, c).  A column of a personalised batch often sums
// thousands of nearly equal small contributions next to one large one; plain sequential FP32
// addition then rounds the same way every time and drifts.
__device__ __forceinline__ void kahan_add(float &sum, float &c, float y) {
    const float yc = y - c;
    const float t = sum + yc;
    c = (t - sum) - yc;
    sum = t;
}

__device__ __forceinline__ void kahan_add4(float4 &sum, float4 &c, float4 y) {
    kahan_add(sum.x, c.x, y.x);
    kahan_add(sum.y, c.y, y.y);
    kahan_add(sum.z, c.z, y.z);
    kahan_add(sum.w, c.w, y.w);
}

__device__ __forceinline__ float4 add4(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }

constexpr int PPR_THREADS = 256;
constexpr int PPR_WARPS = PPR_THREADS / 32;
constexpr double PPR_FX = 2305843009213693952.0;  // 2^61: every column has L1 mass <= 1

// Rows with more than PPR_PIECE in-edges are cut into pieces of PPR_PIECE edges, each summed by
// its own warp into a partial row (k_ppr_piece), and finished by k_ppr_fix, which adds the
// pieces of a row in order: a hub no longer serialises a whole iteration on one warp.
constexpr int PPR_PIECE = 2048;

template <int NV4>
__device__ __forceinline__ void ppr_row_sum(const int32_t *__restrict__ colidx, int32_t s, int32_t e,
                                            const float4 *__restrict__ C, int lane, float4 *acc) {
    constexpr int NP = 128 * NV4;
    constexpr int U = NV4 <= 2 ? 4 : 2;  // rows in flight (a power of two)
    float4 comp[NV4];
#pragma unroll
    for (int q = 0; q < NV4; ++q) comp[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    int32_t i = s;
    for (; i + U - 1 < e; i += U) {
        int64_t u[U];
#pragma unroll
        for (int k2 = 0; k2 < U; ++k2) u[k2] = __ldg(colidx + i + k2);
        float4 x[U][NV4];
#pragma unroll
        for (int k2 = 0; k2 < U; ++k2)
#pragma unroll
            for (int q = 0; q < NV4; ++q) x[k2][q] = __ldg(C + u[k2] * (NP / 4) + 32 * q + lane);
#pragma unroll
        for (int q = 0; q < NV4; ++q) {  // tree sum of the group, then one compensated add
            float4 gsum = add4(x[0][q], x[1][q]);
            if (U == 4) gsum = add4(gsum, add4(x[2][q], x[3][q]));
            kahan_add4(acc[q], comp[q], gsum);
        }
    }
    for (; i < e; ++i) {
        const int64_t u0 = __ldg(colidx + i);
#pragma unroll
        for (int q = 0; q < NV4; ++q) kahan_add4(acc[q], comp[q], __ldg(C + u0 * (NP / 4) + 32 * q + lane));
    }
}

// pieces: (row, first edge) pairs; piece p covers [first, min(first + PPR_PIECE, row end))
template <int NV4>
__global__ void __launch_bounds__(PPR_THREADS) k_ppr_piece(const int32_t *__restrict__ rowptr,
                                                           const int32_t *__restrict__ colidx,
                                                           const int2 *__restrict__ pieces, int32_t npieces,
                                                           const float4 *__restrict__ C, float4 *__restrict__ Ppc) {
    constexpr int NP = 128 * NV4;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * PPR_WARPS;
    for (int64_t p = (int64_t)blockIdx.x * PPR_WARPS + (threadIdx.x >> 5); p < npieces; p += nw) {
        const int2 pc = pieces[p];
        const int32_t e = min(pc.y + PPR_PIECE, __ldg(rowptr + pc.x + 1));
        float4 acc[NV4];
#pragma unroll
        for (int q = 0; q < NV4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        ppr_row_sum<NV4>(colidx, pc.y, e, C, lane, acc);
#pragma unroll
        for (int q = 0; q < NV4; ++q) Ppc[p * (NP / 4) + 32 * q + lane] = acc[q];
    }
}

template <int NV4>  // float4 per lane; columns in the padded batch = 128 * NV4
__global__ void __launch_bounds__(PPR_THREADS) k_ppr_gather(const int32_t *__restrict__ rowptr,
                                                            const int32_t *__restrict__ colidx, int32_t V,
                                                            const float4 *__restrict__ C, float4 *__restrict__ Cn,
                                                            const int32_t *__restrict__ src_of_col,
                                                            const unsigned long long *__restrict__ Dcur,
                                                            unsigned long long *Dnext, unsigned long long *Dzero,
                                                            const float *__restrict__ inv_outdeg, float damping,
                                                            float *R_out, int32_t n,
                                                            const int32_t *__restrict__ hub_rows,
                                                            const int32_t *__restrict__ hub_piece0, int32_t nhubs,
                                                            const float4 *__restrict__ Ppc,
                                                            const uint8_t *__restrict__ is_src) {
    constexpr int NP = 128 * NV4;
    // per-column constants live in shared memory (registers go to rows in flight): the source
    // vertex and teleport term of each column, and each warp's dangling sums
    __shared__ float dsh[PPR_WARPS][NP];
    __shared__ int32_t ssrc[NP];
    __shared__ float stele[NP];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < NP; j += PPR_THREADS) Dzero[j] = 0ull;
    for (int j = threadIdx.x; j < NP; j += PPR_THREADS) {
        ssrc[j] = src_of_col[j];
        stele[j] = (1.0f - damping) + damping * (float)((double)Dcur[j] / PPR_FX);
    }
    for (int j = lane; j < NP; j += 32) dsh[warp][j] = 0.0f;
    __syncthreads();
    const int64_t nw = (int64_t)gridDim.x * PPR_WARPS;
    // the hub rows (finished from their pieces) come first, then every other row
    for (int64_t w = (int64_t)blockIdx.x * PPR_WARPS + warp; w < (int64_t)V + nhubs; w += nw) {
        float4 acc[NV4];
#pragma unroll
        for (int q = 0; q < NV4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t v;
        if (w < nhubs) {
            v = hub_rows[w];
            const int32_t p0 = hub_piece0[w], p1 = hub_piece0[w + 1];
            for (int32_t p = p0; p < p1; ++p)  // pieces in order
#pragma unroll
                for (int q = 0; q < NV4; ++q) {
                    const float4 x = Ppc[(int64_t)p * (NP / 4) + 32 * q + lane];
                    acc[q].x += x.x;
                    acc[q].y += x.y;
                    acc[q].z += x.z;
                    acc[q].w += x.w;
                }
        } else {
            v = w - nhubs;
            const int32_t s = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
            if (e - s > PPR_PIECE) continue;  // a hub: done above
            ppr_row_sum<NV4>(colidx, s, e, C, lane, acc);
        }
        const float inv = __ldg(inv_outdeg + v);
        const bool vsrc = __ldg(is_src + v) != 0;  // the same byte for the whole warp
#pragma unroll
        for (int q = 0; q < NV4; ++q) {
            float r[4] = {acc[q].x, acc[q].y, acc[q].z, acc[q].w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int j = 128 * q + 4 * lane + c;
                r[c] = damping * r[c] + ((vsrc && ssrc[j] == (int32_t)v) ? stele[j] : 0.0f);
                if (inv == 0.0f) dsh[warp][j] += r[c];  // lane-owned columns: no race
            }
            Cn[v * (NP / 4) + 32 * q + lane] = make_float4(r[0] * inv, r[1] * inv, r[2] * inv, r[3] * inv);
            if (R_out) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = 128 * q + 4 * lane + c;
                    if (j < n) R_out[v * n + j] = r[c];
                }
            }
        }
    }
    // per-column dangling sums: warps -> shared -> one fixed-point atomic per column per CTA
    __syncthreads();
    for (int j = threadIdx.x; j < NP; j += PPR_THREADS) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < PPR_WARPS; ++w) t += dsh[w][j];
        if (t != 0.0f) atomicAdd(Dnext + j, (unsigned long long)__double2ll_rn((double)t * PPR_FX));
    }
}

// C = e_{s_j} scaled by 1/out_degree(s_j); D0_j = [s_j dangling]; optional R_out = e_{s_j}.
__global__ void k_ppr_init(float *C, int32_t NP, const int32_t *src_of_col, const float *inv_outdeg,
                           unsigned long long *D0, float *R_out, int32_t n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NP; j += gridDim.x * blockDim.x) {
        const int32_t s = src_of_col[j];
        D0[j] = 0ull;
        if (s < 0) continue;
        const float inv = inv_outdeg[s];
        C[(int64_t)s * NP + j] = inv;
        if (inv == 0.0f) D0[j] = (unsigned long long)PPR_FX;
        if (R_out && j < n) R_out[(int64_t)s * n + j] = 1.0f;
    }
}

// ---------------------------------------------------------------------------------------------
// TOCAB form of the batch (Sec. 3.1 applied to a column tile): the n columns are processed in
// tiles of 32; for tile t the contribution matrix is read as 128-byte row segments C[u, 32t..]
// and the pull partition's source blocks are sized so that one block's segments stay in L2.
// Alg. 4 per block writes 32-wide partial rows; the merge of Fig. 5 (CTA per vertex range, the
// blocks added in block order - deterministic) applies the update for the tile's columns.
// ---------------------------------------------------------------------------------------------
constexpr int PT_THREADS = 256;
constexpr int PT_WARPS = PT_THREADS / 32;

constexpr int PT_PIECE = 1024;  // local rows above this many edges are cut into pieces

// Edges [s, e) of one row, tile t: 8 lanes (sub) each summing one float4 of the 32 columns.
__device__ __forceinline__ float4 tile_row_sum(const int32_t *__restrict__ colidx, int32_t s, int32_t e,
                                               const float4 *__restrict__ Ct, int64_t NP4) {
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), c = a;
    int32_t i = s;
    for (; i + 3 < e; i += 4) {
        const int64_t u0 = __ldg(colidx + i), u1 = __ldg(colidx + i + 1), u2 = __ldg(colidx + i + 2),
                      u3 = __ldg(colidx + i + 3);
        const float4 x0 = __ldg(Ct + u0 * NP4), x1 = __ldg(Ct + u1 * NP4), x2 = __ldg(Ct + u2 * NP4),
                     x3 = __ldg(Ct + u3 * NP4);
        kahan_add4(a, c, add4(add4(x0, x1), add4(x2, x3)));
    }
    for (; i < e; ++i) kahan_add4(a, c, __ldg(Ct + (int64_t)__ldg(colidx + i) * NP4));
    return a;
}

// pieces of long local rows: 4 pieces per warp, 8 lanes each -> partial rows Ppc[piece][32]
__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_piece(const int32_t *__restrict__ rowptr,
                                                               const int32_t *__restrict__ colidx,
                                                               const int2 *__restrict__ pieces, int32_t npieces,
                                                               const float *__restrict__ C, int32_t NP, int32_t t,
                                                               float *__restrict__ Ppc) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7, slot = lane >> 3;
    const int64_t nw = (int64_t)gridDim.x * PT_WARPS;
    const float4 *Ct = reinterpret_cast<const float4 *>(C + 32 * t) + sub;
    for (int64_t p0 = ((int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5)) * 4; p0 < npieces; p0 += nw * 4) {
        const int64_t p = p0 + slot;
        int32_t s = 0, e = 0;
        if (p < npieces) {
            const int2 pc = pieces[p];
            s = pc.y;
            e = min(pc.y + PT_PIECE, __ldg(rowptr + pc.x + 1));
        }
        const float4 a = tile_row_sum(colidx, s, e, Ct, NP / 4);
        if (p < npieces) reinterpret_cast<float4 *>(Ppc)[p * 8 + sub] = a;
    }
}

// long rows: P[row] = sum of the row's pieces, in order
__global__ void k_ppr_tile_fix(const int32_t *__restrict__ hub_rows, const int32_t *__restrict__ piece0, int32_t nh,
                               const float *__restrict__ Ppc, float *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t h = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; h < nh; h += nw) {
        float a = 0.0f;
        for (int32_t p = piece0[h]; p < piece0[h + 1]; ++p) a += Ppc[(int64_t)p * 32 + lane];
        P[(int64_t)hub_rows[h] * 32 + lane] = a;
    }
}

// Four rows per warp: 8 lanes per row, one float4 each (the tile's 32 columns = 128 bytes), and
// four in-edges in flight per row, so that every warp keeps 16 segment loads outstanding.
__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_gather(const int32_t *__restrict__ rowptr,
                                                                const int32_t *__restrict__ colidx, int64_t R,
                                                                const float *__restrict__ C, int32_t NP, int32_t t,
                                                                float *__restrict__ P) {
    const int lane = threadIdx.x & 31;
    const int sub = lane & 7, slot = lane >> 3;  // 4 rows per warp, 8 lanes per row
    const int64_t nw = (int64_t)gridDim.x * PT_WARPS;
    const float4 *Ct = reinterpret_cast<const float4 *>(C + 32 * t) + sub;
    const int64_t NP4 = NP / 4;
    for (int64_t r0 = ((int64_t)blockIdx.x * PT_WARPS + (threadIdx.x >> 5)) * 4; r0 < R; r0 += nw * 4) {
        const int64_t r = r0 + slot;
        int32_t s = 0, e = 0;
        if (r < R) {
            s = __ldg(rowptr + r);
            e = __ldg(rowptr + r + 1);
        }
        const bool longrow = e - s > PT_PIECE;  // finished from its pieces
        const float4 a = tile_row_sum(colidx, s, longrow ? s : e, Ct, NP4);
        if (r < R && !longrow) reinterpret_cast<float4 *>(P)[r * 8 + sub] = a;
    }
}

__global__ void __launch_bounds__(PT_THREADS) k_ppr_tile_merge(const float *__restrict__ P,
                                                               const int32_t *__restrict__ id_map,
                                                               const int32_t *__restrict__ merge_off, int32_t B,
                                                               int32_t nranges, int32_t k, int32_t V, int32_t NP,
                                                               int32_t t, const int32_t *__restrict__ src_of_col,
                                                               const unsigned long long *__restrict__ Dcur,
                                                               unsigned long long *Dnext, unsigned long long *Dzero,
                                                               const float *__restrict__ inv_outdeg, float damping,
                                                               float *Cn, float *R_out, int32_t n) {
    extern __shared__ float pacc[];  // [k][32]
    __shared__ float dsh[PT_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int32_t j = blockIdx.x;
    const int32_t vbase = j * k;
    if (blockIdx.x == 0 && t == 0)
        for (int q = threadIdx.x; q < NP; q += PT_THREADS) Dzero[q] = 0ull;
    for (int q = threadIdx.x; q < k * 32; q += PT_THREADS) pacc[q] = 0.0f;
    __syncthreads();
    for (int32_t b = 0; b < B; ++b) {  // blocks in order: every vertex's sum has a fixed order
        const int32_t *o = merge_off + (int64_t)b * (nranges + 1) + j;
        const int32_t r0 = __ldg(o), r1 = __ldg(o + 1);
        for (int32_t r = r0 + warp; r < r1; r += PT_WARPS)
            pacc[(__ldg(id_map + r) - vbase) * 32 + lane] += __ldg(P + (int64_t)r * 32 + lane);
        __syncthreads();
    }
    const int32_t col = 32 * t + lane;
    const int32_t s = src_of_col[col];
    const float tele = (1.0f - damping) + damping * (float)((double)Dcur[col] / PPR_FX);
    float dl = 0.0f;
    for (int32_t q = warp; q < k; q += PT_WARPS) {
        const int32_t v = vbase + q;
        if (v >= V) break;
        const float r = damping * pacc[q * 32 + lane] + (s == v ? tele : 0.0f);
        const float inv = __ldg(inv_outdeg + v);
        Cn[(int64_t)v * NP + col] = r * inv;
        if (R_out && col < n) R_out[(int64_t)v * n + col] = r;
        if (inv == 0.0f) dl += r;
    }
    dsh[warp][lane] = dl;
    __syncthreads();
    if (warp == 0) {
        float tot = 0.0f;
#pragma unroll
        for (int w = 0; w < PT_WARPS; ++w) tot += dsh[w][lane];
        if (tot != 0.0f) atomicAdd(Dnext + col, (unsigned long long)__double2ll_rn((double)tot * PPR_FX));
    }
}

__global__ void k_mark_sources(const int32_t *src_of_col, int32_t NP, uint8_t *is_src) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < NP; j += gridDim.x * blockDim.x)
        if (src_of_col[j] >= 0) is_src[src_of_col[j]] = 1;
}

struct Hubs {
    const int32_t *rows, *piece0;
    const int2 *pieces;
    int32_t nhubs, npieces;
    float *Ppc;
};

template <int NV4>
static void launch_ppr(int grid, cudaStream_t s, const tc_graph *g, const float *C, float *Cn, const int32_t *srcc,
                       const unsigned long long *Dc, unsigned long long *Dn, unsigned long long *Dz, float d,
                       float *R_out, int32_t n, const Hubs &h, const uint8_t *is_src) {
    if (h.npieces > 0)
        k_ppr_piece<NV4><<<grid, PPR_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), h.pieces,
                                                     h.npieces, reinterpret_cast<const float4 *>(C),
                                                     reinterpret_cast<float4 *>(h.Ppc));
    k_ppr_gather<NV4><<<grid, PPR_THREADS, 0, s>>>(g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), g->V,
                                                  reinterpret_cast<const float4 *>(C), reinterpret_cast<float4 *>(Cn),
                                                  srcc, Dc, Dn, Dz, g->inv_outdeg.as<float>(), d, R_out, n, h.rows,
                                                  h.piece0, h.nhubs, reinterpret_cast<const float4 *>(h.Ppc), is_src);
}

__global__ void k_row_bounds(const int32_t *rowptr, const int32_t *rows, int32_t n, int32_t *out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[2 * i] = rowptr[rows[i]];
        out[2 * i + 1] = rowptr[rows[i] + 1];
    }
}

// Pieces of the rows above `piece` edges: host-built from the hub list (few rows).
static int build_pieces(const int32_t *rowptr, const int32_t *hub_list, int32_t nh, int32_t NP, DevBuf *rows,
                        DevBuf *piece0, DevBuf *pieces, DevBuf *Ppc, Hubs *h, cudaStream_t s,
                        int32_t piece = PPR_PIECE) {
    h->nhubs = 0;
    h->npieces = 0;
    h->rows = nullptr;
    h->piece0 = nullptr;
    h->pieces = nullptr;
    h->Ppc = nullptr;
    if (nh <= 0) return TC_OK;
    int32_t *hl = new (std::nothrow) int32_t[nh];
    int32_t *rs = new (std::nothrow) int32_t[2 * (size_t)nh];
    if (!hl || !rs) {
        delete[] hl;
        delete[] rs;
        return fail(TC_ERR_OOM, "host allocation failed");
    }
    DevBuf bounds;
    int brc = bounds.alloc((size_t)nh * 8);
    if (brc != TC_OK) {
        delete[] hl;
        delete[] rs;
        return brc;
    }
    k_row_bounds<<<(nh + 255) / 256, 256, 0, s>>>(rowptr, hub_list, nh, bounds.as<int32_t>());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hl, hub_list, (size_t)nh * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rs, bounds.p, (size_t)nh * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        delete[] hl;
        delete[] rs;
        return fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    }
    int32_t *p0 = new (std::nothrow) int32_t[nh + 1];
    int64_t np = 0;
    for (int32_t i = 0; i < nh; ++i) np += (rs[2 * i + 1] - rs[2 * i] + piece - 1) / piece;
    int2 *pc = new (std::nothrow) int2[np > 0 ? np : 1];
    if (!p0 || !pc) {
        delete[] hl;
        delete[] rs;
        delete[] p0;
        delete[] pc;
        return fail(TC_ERR_OOM, "host allocation failed");
    }
    int64_t q = 0;
    for (int32_t i = 0; i < nh; ++i) {
        p0[i] = (int32_t)q;
        for (int32_t st = rs[2 * i]; st < rs[2 * i + 1]; st += piece) pc[q++] = make_int2(hl[i], st);
    }
    p0[nh] = (int32_t)q;
    int rc = rows->alloc((size_t)nh * 4);
    if (rc == TC_OK) rc = piece0->alloc((size_t)(nh + 1) * 4);
    if (rc == TC_OK) rc = pieces->alloc((size_t)(np > 0 ? np : 1) * 8);
    if (rc == TC_OK) rc = Ppc->alloc((size_t)(np > 0 ? np : 1) * NP * 4);
    if (rc == TC_OK) {
        e = cudaMemcpyAsync(rows->p, hl, (size_t)nh * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(piece0->p, p0, (size_t)(nh + 1) * 4, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pieces->p, pc, (size_t)np * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    }
    delete[] hl;
    delete[] rs;
    delete[] p0;
    delete[] pc;
    if (rc != TC_OK) return rc;
    h->nhubs = nh;
    h->npieces = (int32_t)np;
    h->rows = rows->as<int32_t>();
    h->piece0 = piece0->as<int32_t>();
    h->pieces = pieces->as<int2>();
    h->Ppc = Ppc->as<float>();
    return TC_OK;
}

static int ppr_impl(const tc_graph *cg, const tc_part *part, const int32_t *sources, int32_t n,
                    const tc_pr_params *pp, float *R_out, tc_pr_stats *stats, cudaStream_t s) {
    tc_graph *g = const_cast<tc_graph *>(cg);
    const int32_t V = g->V;
    int NV4 = 1;
    while (128 * NV4 < n) NV4 *= 2;
    const int32_t NP = 128 * NV4;
    const size_t mat = (size_t)V * NP * 4;
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    DevBuf Cbuf, srcbuf, Dbuf, Rdev;
    TC_TRY(Cbuf.alloc(2 * mat));
    TC_TRY(srcbuf.alloc((size_t)NP * 4));
    TC_TRY(Dbuf.alloc((size_t)3 * NP * 8));
    float *Cm[2] = {Cbuf.as<float>(), Cbuf.as<float>() + (size_t)V * NP};
    unsigned long long *D[3] = {Dbuf.as<unsigned long long>(), Dbuf.as<unsigned long long>() + NP,
                                Dbuf.as<unsigned long long>() + 2 * NP};
    int32_t *hsrc = new (std::nothrow) int32_t[NP];
    if (!hsrc) return fail(TC_ERR_OOM, "host allocation failed");
    for (int32_t j = 0; j < NP; ++j) hsrc[j] = j < n ? sources[j] : -1;
    cudaError_t e = cudaMemcpyAsync(srcbuf.p, hsrc, (size_t)NP * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] hsrc;
    if (e != cudaSuccess) return fail(TC_ERR_CUDA, "tc_ppr_batch: %s", cudaGetErrorString(e));
    float *Rd = R_out;
    if (pp->out_mem == TC_MEM_HOST) {
        TC_TRY(Rdev.alloc((size_t)V * n * 4));
        Rd = Rdev.as<float>();
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (pp->profile) {
        TC_CUDA(cudaEventCreate(&ev[0]));
        TC_CUDA(cudaEventCreate(&ev[1]));
        TC_CUDA(cudaEventRecord(ev[0], s));
    }
    TC_CUDA(cudaMemsetAsync(Cm[0], 0, mat, s));
    if (pp->iters == 0) TC_CUDA(cudaMemsetAsync(Rd, 0, (size_t)V * n * 4, s));
    k_ppr_init<<<(NP + 255) / 256, 256, 0, s>>>(Cm[0], NP, srcbuf.as<int32_t>(), g->inv_outdeg.as<float>(), D[0],
                                                pp->iters == 0 ? Rd : nullptr, n);
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaMemsetAsync(D[1], 0, (size_t)NP * 8, s));
    int per_sm = 1;
    const void *kf = NV4 == 1 ? (const void *)k_ppr_gather<1>
                     : NV4 == 2 ? (const void *)k_ppr_gather<2>
                     : NV4 == 4 ? (const void *)k_ppr_gather<4>
                                : (const void *)k_ppr_gather<8>;
    TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kf, PPR_THREADS, 0));
    const int grid = caps.sms * (per_sm > 0 ? per_sm : 1);
    int launches = 1;
    const int32_t ntiles = NP / 32;
    DevBuf Pbuf;
    size_t tm_smem = 0;
    int tg_grid = 1;
    Hubs th;
    DevBuf th_list, th_rows, th_p0, th_pcs, th_ppc;
    int32_t tnh = 0;
    if (part) {
        TC_TRY(collect_hubs(part->rowptr.as<int32_t>(), part->R, PT_PIECE, &th_list, &tnh, s));
        // piece partials are 32 floats: NP argument 32
        TC_TRY(build_pieces(part->rowptr.as<int32_t>(), th_list.as<int32_t>(), tnh, 32, &th_rows, &th_p0, &th_pcs,
                            &th_ppc, &th, s, PT_PIECE));
        TC_TRY(Pbuf.alloc((size_t)(part->R > 0 ? part->R : 1) * 32 * 4));
        tm_smem = (size_t)part->k * 32 * 4;
        TC_CUDA(cudaFuncSetAttribute(k_ppr_tile_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tm_smem));
        int ps = 1;
        TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_ppr_tile_gather, PT_THREADS, 0));
        tg_grid = caps.sms * (ps > 0 ? ps : 1);
    }
    for (int it = 0; it < pp->iters && part; ++it) {
        const bool last = it == pp->iters - 1;
        const float *Cc = Cm[it & 1];
        float *Cn = Cm[(it + 1) & 1];
        unsigned long long *Dc = D[it % 3], *Dn = D[(it + 1) % 3], *Dz = D[(it + 2) % 3];
        for (int32_t t = 0; t < ntiles; ++t) {
            if (th.npieces > 0) {
                k_ppr_tile_piece<<<tg_grid, PT_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                                th.pieces, th.npieces, Cc, NP, t, th.Ppc);
                ++launches;
            }
            k_ppr_tile_gather<<<tg_grid, PT_THREADS, 0, s>>>(part->rowptr.as<int32_t>(), part->colidx.as<int32_t>(),
                                                             part->R, Cc, NP, t, Pbuf.as<float>());
            if (th.nhubs > 0) {
                k_ppr_tile_fix<<<(th.nhubs * 32 + 255) / 256, 256, 0, s>>>(th.rows, th.piece0, th.nhubs, th.Ppc,
                                                                          Pbuf.as<float>());
                ++launches;
            }
            k_ppr_tile_merge<<<part->nranges, PT_THREADS, tm_smem, s>>>(
                Pbuf.as<float>(), part->id_map.as<int32_t>(), part->merge_off.as<int32_t>(), part->B, part->nranges,
                part->k, g->V, NP, t, srcbuf.as<int32_t>(), Dc, Dn, Dz, g->inv_outdeg.as<float>(), pp->damping,
                Cn, last ? Rd : nullptr, n);
            TC_LAUNCH_CHECK();
            launches += 2;
        }
    }
    Hubs hubs;
    DevBuf hub_list, hub_rows, hub_p0, hub_pcs, hub_ppc, isrc;
    int32_t nh = 0;
    if (!part) {
        // one byte per vertex: 1 where some column teleports to it
        TC_TRY(isrc.alloc((size_t)V));
        TC_CUDA(cudaMemsetAsync(isrc.p, 0, (size_t)V, s));
        k_mark_sources<<<(NP + 255) / 256, 256, 0, s>>>(srcbuf.as<int32_t>(), NP, isrc.as<uint8_t>());
        TC_LAUNCH_CHECK();
        TC_TRY(collect_hubs(g->in_rowptr.as<int32_t>(), g->V, PPR_PIECE, &hub_list, &nh, s));
        TC_TRY(build_pieces(g->in_rowptr.as<int32_t>(), hub_list.as<int32_t>(), nh, NP, &hub_rows, &hub_p0, &hub_pcs,
                            &hub_ppc, &hubs, s));
    }
    for (int it = 0; it < pp->iters && !part; ++it) {
        const bool last = it == pp->iters - 1;
        float *Rw = last ? Rd : nullptr;
        const float *Cc = Cm[it & 1];
        float *Cn = Cm[(it + 1) & 1];
        unsigned long long *Dc = D[it % 3], *Dn = D[(it + 1) % 3], *Dz = D[(it + 2) % 3];
        switch (NV4) {
            case 1: launch_ppr<1>(grid, s, g, Cc, Cn, srcbuf.as<int32_t>(), Dc, Dn, Dz, pp->damping, Rw, n, hubs,
                                    isrc.as<uint8_t>()); break;
            case 2: launch_ppr<2>(grid, s, g, Cc, Cn, srcbuf.as<int32_t>(), Dc, Dn, Dz, pp->damping, Rw, n, hubs,
                                    isrc.as<uint8_t>()); break;
            case 4: launch_ppr<4>(grid, s, g, Cc, Cn, srcbuf.as<int32_t>(), Dc, Dn, Dz, pp->damping, Rw, n, hubs,
                                    isrc.as<uint8_t>()); break;
            default: launch_ppr<8>(grid, s, g, Cc, Cn, srcbuf.as<int32_t>(), Dc, Dn, Dz, pp->damping, Rw, n, hubs,
                                    isrc.as<uint8_t>()); break;
        }
        TC_LAUNCH_CHECK();
        ++launches;
    }
    float ms = 0;
    if (pp->profile) {
        TC_CUDA(cudaEventRecord(ev[1], s));
        TC_CUDA(cudaEventSynchronize(ev[1]));
        TC_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
        cudaEventDestroy(ev[0]);
        cudaEventDestroy(ev[1]);
    }
    if (pp->out_mem == TC_MEM_HOST)
        TC_CUDA(cudaMemcpyAsync(R_out, Rd, (size_t)V * n * 4, cudaMemcpyDeviceToHost, s));
    // the scratch buffers are freed at return: finish their users first
    TC_CUDA(cudaStreamSynchronize(s));
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->iters = pp->iters;
        stats->launches = launches;
        stats->ms_total = ms;
        stats->ms_gather = ms;
    }
    return TC_OK;
}

}  // namespace tc

extern "C" int tc_ppr_batch(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t n,
                            const tc_pr_params *params, float *R_out, tc_pr_stats *stats, void *stream) {
    using namespace tc;
    if (!g || !sources || !params || !R_out) return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: null argument");
    if (part && (part->g != g || part->dir != TC_PULL))
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: partition must be a TC_PULL partition of this graph");
    if (part && part->order != TC_ORDER_NATURAL)
        return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: renumbered (TC_ORDER_OUTDEGREE) partitions are not supported");
    if (part && (size_t)part->k * 32 * 4 > 200 * 1024)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: the partition's merge_range must be <= 1600 (<= 256 advised)");
    if (n < 1 || n > 1024) return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: n must be in [1, 1024]");
    if (!(params->damping >= 0.0f && params->damping <= 1.0f) || params->iters < 0)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: damping outside [0,1] or iters < 0");
    if (params->out_mem != TC_MEM_HOST && params->out_mem != TC_MEM_DEVICE)
        return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: bad out_mem");
    for (int32_t j = 0; j < n; ++j)
        if (sources[j] < 0 || sources[j] >= g->V) return fail(TC_ERR_INVALID_ARG, "tc_ppr_batch: source %d outside [0, V)", j);
    if ((int64_t)g->V * ((n + 127) / 128 * 128) * 8 > ((int64_t)1 << 40))
        return fail(TC_ERR_UNSUPPORTED, "tc_ppr_batch: V x n too large");
    return ppr_impl(g, part, sources, n, params, R_out, stats, (cudaStream_t)stream);
}
