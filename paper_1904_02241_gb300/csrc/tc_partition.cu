// TOCAB preprocessing (Sec. 3.1): static 1D blocking of a CSR by column ranges, local IDs
// for the rows that have edges in a block (Fig. 4), the merge range table (Fig. 5) and the
// hub-row list used by the load balancer (Sec. 3.2).  Everything runs on the device.
#include "tc_internal.cuh"

namespace tc {

// head[i] = 1 when edge i starts a new local row: first edge, new block or new row.
__global__ void k_row_heads(const int32_t *col, const int32_t *row, int64_t E, DivBy W, uint8_t *head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E; i += (int64_t)gridDim.x * blockDim.x) {
        bool h = true;
        if (i > 0) h = (div_apply(col[i], W) != div_apply(col[i - 1], W)) || (row[i] != row[i - 1]);
        head[i] = h ? 1 : 0;
    }
}

// blk_edges[b] = first edge whose column is >= b*W (columns are block-major after the sort);
// blk_rows[b] = the local row starting at that edge (every block starts a row), R past the end.
__global__ void k_block_bounds(const int32_t *col, const int32_t *rowptr, int64_t E, int64_t R, int32_t W, int32_t B,
                               int64_t *blk_edges, int64_t *blk_rows) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b <= B; b += gridDim.x * blockDim.x) {
        const int64_t bound = (int64_t)b * W;
        int64_t lo = 0, hi = E;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)col[mid] < bound) lo = mid + 1; else hi = mid;
        }
        blk_edges[b] = lo;
        int64_t rl = 0, rh = R;  // first row whose first edge is >= lo
        while (rl < rh) {
            const int64_t mid = (rl + rh) >> 1;
            if ((int64_t)rowptr[mid] < lo) rl = mid + 1; else rh = mid;
        }
        blk_rows[b] = rl;
    }
}

// off[b][j] = first local row of block b whose global id is >= the first vertex of merge range
// j (j*k, or rstart[j] when the ranges are given), j in [0, nranges]; offT[j][b] holds the same
// table range-major (the merge of range j reads one row of it).
__global__ void k_merge_offsets(const int32_t *id_map, const int64_t *blk_rows, int32_t B, int32_t nranges, int32_t k,
                                const int32_t *rstart, int32_t *off, int32_t *offT) {
    const int64_t total = (int64_t)B * (nranges + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = (int32_t)(t / (nranges + 1));
        const int32_t j = (int32_t)(t - (int64_t)b * (nranges + 1));
        const int64_t bound = rstart ? (int64_t)rstart[j] : (int64_t)j * k;
        int64_t lo = blk_rows[b], hi = blk_rows[b + 1];
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if ((int64_t)id_map[mid] < bound) lo = mid + 1; else hi = mid;
        }
        off[t] = (int32_t)lo;
        offT[(int64_t)j * B + b] = (int32_t)lo;
    }
}

// gpre[j][b] = granules (aligned groups of MERGE_GRAN local rows that hold rows of the slice)
// in the slices of blocks 0..b-1 of merge range j; gpre[j][B] = all of range j's.  One CTA per
// range (grid-stride), an exclusive scan over the blocks in chunks of the CTA's width.
__global__ void __launch_bounds__(256) k_merge_gpre(const int32_t *offT, int32_t B, int32_t nranges, int32_t *gpre) {
    __shared__ int32_t wsum[8];
    __shared__ int32_t carry_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int32_t j = blockIdx.x; j < nranges; j += gridDim.x) {
        int32_t carry = 0;
        for (int32_t b0 = 0; b0 < B; b0 += 256) {
            const int32_t b = b0 + tid;
            int32_t cnt = 0;
            if (b < B) {
                const int32_t l0 = offT[(int64_t)j * B + b], l1 = offT[(int64_t)(j + 1) * B + b];
                cnt = l1 > l0 ? (l1 + MERGE_GRAN - 1) / MERGE_GRAN - l0 / MERGE_GRAN : 0;
            }
            int32_t incl = cnt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();
            int32_t before = carry;
            for (int w = 0; w < warp; ++w) before += wsum[w];
            if (b < B) gpre[(int64_t)j * (B + 1) + b] = before + incl - cnt;
            if (tid == 255) carry_s = before + incl;
            __syncthreads();
            carry = carry_s;
            __syncthreads();
        }
        if (tid == 0) gpre[(int64_t)j * (B + 1) + B] = carry;
    }
}

__global__ void k_id16(const int32_t *id_map, int64_t R, int32_t kmask, uint16_t *id16) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
        id16[r] = (uint16_t)(id_map[r] & kmask);
}

// id16[r] = id_map[r] minus the first vertex of its merge range (the last rstart <= the id).
__global__ void k_id16_ranges(const int32_t *id_map, int64_t R, const int32_t *rstart, int32_t nranges,
                              uint16_t *id16) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = id_map[r];
        int32_t lo = 0, hi = nranges - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (rstart[mid] <= v) lo = mid; else hi = mid - 1;
        }
        id16[r] = (uint16_t)(v - rstart[lo]);
    }
}

// ---- vertex renumbering by out-degree (TC_ORDER_OUTDEGREE) ---------------------------------
// key[v] = maxdeg - out_degree(v), or maxdeg + 1 for a vertex without any edge: an ascending
// stable sort of the keys lists the vertices by out-degree, highest first, ties in ID order, with
// the vertices that have no edge at all after those that have in-edges only.  *isolated counts
// the vertices without any edge.
__global__ void k_order_keys(const int32_t *out_rowptr, const int32_t *in_rowptr, int32_t V, int32_t maxdeg,
                             int32_t *key, int32_t *val, int32_t *isolated) {
    int32_t n = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t od = out_rowptr[v + 1] - out_rowptr[v];
        const bool iso = od == 0 && in_rowptr[v + 1] == in_rowptr[v];
        key[v] = iso ? maxdeg + 1 : maxdeg - od;
        val[v] = (int32_t)v;
        n += iso;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n += __shfl_xor_sync(0xffffffffu, n, d);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(isolated, n);
}

// For new vertex n with original ID perm[n]: inv[perm[n]] = n, its in-degree (row length of the
// renumbered G^T; deg[V] = 0 closes the scan) and its out-degree reciprocal.
__global__ void k_order_apply(const int32_t *perm, const int32_t *in_rowptr, const float *inv_outdeg_old, int32_t V,
                              int32_t *inv, int32_t *deg, float *inv_outdeg_new) {
    for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n <= V; n += (int64_t)gridDim.x * blockDim.x) {
        if (n == V) {
            deg[V] = 0;
            continue;
        }
        const int32_t o = perm[n];
        inv[o] = (int32_t)n;
        deg[n] = in_rowptr[o + 1] - in_rowptr[o];
        inv_outdeg_new[n] = inv_outdeg_old[o];
    }
}

// Renumbered G^T: edge e of new row n is edge (e - rowptr_new[n]) of old row perm[n], with its
// source renumbered.  Sources keep the old row's order (ascending old ID).
__global__ void k_order_edges(const int32_t *row_of_edge, const int32_t *rowptr_new, const int32_t *perm,
                              const int32_t *in_rowptr, const int32_t *in_colidx, const int32_t *inv, int64_t E,
                              int32_t *colidx_new) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t n = row_of_edge[e];
        const int64_t src_pos = (int64_t)in_rowptr[perm[n]] + (e - rowptr_new[n]);
        colidx_new[e] = inv[in_colidx[src_pos]];
    }
}

// Pieces per destination: cnt[id_map[r]] += 1 over all local rows.
__global__ void k_pieces_per_vertex(const int32_t *id_map, int64_t R, int32_t *cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + id_map[r], 1);
}

// w[v] = cnt[v] + c for v < V, w[V] = 0 (in place).
__global__ void k_range_weights(int32_t *w, int32_t V, int32_t c) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= V; v += (int64_t)gridDim.x * blockDim.x)
        w[v] = v < V ? w[v] + c : 0;
}

// rstart[j] = the first vertex whose exclusive weight prefix reaches j * total / nr, rounded down
// to a multiple of 32; rstart[0] = 0 and rstart[nr] = V.
__global__ void k_range_bounds(const int64_t *cum /* [V+1] exclusive prefix */, int32_t V, int32_t nr,
                               int32_t *rstart) {
    const int64_t total = cum[V];
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= nr; j += gridDim.x * blockDim.x) {
        if (j == 0 || j == nr) {
            rstart[j] = j == 0 ? 0 : V;
            continue;
        }
        const int64_t target = total * j / nr;  // total < 2^34, nr < 2^20: no overflow
        int64_t lo = 0, hi = V;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (cum[mid] < target) lo = mid + 1; else hi = mid;
        }
        rstart[j] = (int32_t)(lo & ~31LL);
    }
}

__global__ void k_hub_flags(const int32_t *rowptr, int64_t nrows, int32_t min_degree, int32_t *flag) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = (rowptr[r + 1] - rowptr[r]) > min_degree;
}

__global__ void k_hub_compact(const int32_t *flag, const int64_t *pos, int64_t nrows, int32_t *list) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) list[pos[r]] = (int32_t)r;
}

int collect_hubs(const int32_t *rowptr, int64_t nrows, int32_t min_degree, DevBuf *list, int32_t *count,
                 cudaStream_t s) {
    *count = 0;
    if (nrows <= 0) return list->alloc(16);
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    DevBuf flag, pos;
    TC_TRY(flag.alloc(nrows * 4));
    TC_TRY(pos.alloc(nrows * 8));
    k_hub_flags<<<caps.sms * 8, 256, 0, s>>>(rowptr, nrows, min_degree, flag.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32_to_i64(flag.as<int32_t>(), nrows, pos.as<int64_t>(), s));
    int64_t last_pos = 0;
    int32_t last_flag = 0;
    TC_CUDA(cudaMemcpyAsync(&last_pos, pos.as<int64_t>() + nrows - 1, 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(&last_flag, flag.as<int32_t>() + nrows - 1, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    const int64_t n = last_pos + last_flag;
    TC_TRY(list->alloc((n > 0 ? n : 1) * 4));
    if (n > 0) {
        k_hub_compact<<<caps.sms * 8, 256, 0, s>>>(flag.as<int32_t>(), pos.as<int64_t>(), nrows, list->as<int32_t>());
        TC_LAUNCH_CHECK();
    }
    TC_CUDA(cudaStreamSynchronize(s));
    *count = (int32_t)n;
    return TC_OK;
}

static int log2_ceil(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) ++b;
    return b;
}

// Renumber the vertices by out-degree (highest first, ties by ID) and build G^T in the new
// numbering (rp_new, ci_new), the permutation p->perm (new -> old) and the out-degree
// reciprocals p->inv_outdeg in the new order.  Vertices with out-edges get the IDs [0, nz_out).
int order_by_outdegree(const tc_graph *g, cudaStream_t s, DevBuf *perm, DevBuf *inv, DevBuf *inv_outdeg,
                       DevBuf *rp_new, DevBuf *ci_new, DevBuf *row, int32_t *ni) {
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    const int grid = caps.sms * 8;
    const int32_t V = g->V;
    const int64_t E = g->E;
    DevBuf key, val, kout, ktmp, vtmp, deg, niso, row_local;
    TC_TRY(niso.alloc(16));
    TC_CUDA(cudaMemsetAsync(niso.p, 0, 4, s));
    TC_TRY(key.alloc((size_t)V * 4));
    TC_TRY(val.alloc((size_t)V * 4));
    TC_TRY(kout.alloc((size_t)V * 4));
    TC_TRY(ktmp.alloc((size_t)V * 4));
    TC_TRY(vtmp.alloc((size_t)V * 4));
    TC_TRY(perm->alloc((size_t)V * 4));
    TC_TRY(inv_outdeg->alloc((size_t)V * 4 + 256));
    k_order_keys<<<grid, 256, 0, s>>>(g->out_rowptr.as<int32_t>(), g->in_rowptr.as<int32_t>(), V, g->max_out_degree,
                                      key.as<int32_t>(), val.as<int32_t>(), niso.as<int32_t>());
    TC_LAUNCH_CHECK();
    int32_t h_iso = 0;
    TC_CUDA(cudaMemcpyAsync(&h_iso, niso.p, 4, cudaMemcpyDeviceToHost, s));
    TC_TRY(stable_bucket_sort(key.as<int32_t>(), val.as<int32_t>(), kout.as<int32_t>(), perm->as<int32_t>(),
                              ktmp.as<int32_t>(), vtmp.as<int32_t>(), V, 1, log2_ceil((int64_t)g->max_out_degree + 2),
                              s));  // synchronises: h_iso is in
    key.release();
    val.release();
    kout.release();
    ktmp.release();
    vtmp.release();
    TC_TRY(inv->alloc((size_t)V * 4));
    TC_TRY(deg.alloc(((size_t)V + 1) * 4));
    k_order_apply<<<grid, 256, 0, s>>>(perm->as<int32_t>(), g->in_rowptr.as<int32_t>(), g->inv_outdeg.as<float>(), V,
                                       inv->as<int32_t>(), deg.as<int32_t>(), inv_outdeg->as<float>());
    TC_LAUNCH_CHECK();
    TC_TRY(rp_new->alloc(((size_t)V + 1) * 4));
    TC_TRY(scan_i32(deg.as<int32_t>(), (int64_t)V + 1, rp_new->as<int32_t>(), s));
    deg.release();
    TC_TRY(ci_new->alloc((size_t)(E > 0 ? E : 1) * 4));
    if (E > 0) {
        DevBuf *r = row ? row : &row_local;  // the row of every edge of the renumbered G^T
        TC_TRY(r->alloc((size_t)E * 4));
        TC_TRY(expand_rows(rp_new->as<int32_t>(), V, r->as<int32_t>(), s));
        k_order_edges<<<grid, 256, 0, s>>>(r->as<int32_t>(), rp_new->as<int32_t>(), perm->as<int32_t>(),
                                           g->in_rowptr.as<int32_t>(), g->in_colidx.as<int32_t>(), inv->as<int32_t>(), E,
                                           ci_new->as<int32_t>());
        TC_LAUNCH_CHECK();
    }
    TC_CUDA(cudaStreamSynchronize(s));
    *ni = V - h_iso;
    return TC_OK;
}

static int renumber_by_outdegree(const tc_graph *g, cudaStream_t s, DevBuf *rp_new, DevBuf *ci_new, DevBuf *row,
                                 tc_part *p) {
    DevBuf inv;
    int32_t ni = 0;
    TC_TRY(order_by_outdegree(g, s, &p->perm, &inv, &p->inv_outdeg, rp_new, ci_new, row, &ni));
    p->nz_out = (int32_t)((int64_t)g->V - g->num_dangling);
    p->ni = ni;
    p->order = TC_ORDER_OUTDEGREE;
    return TC_OK;
}

// smem_stage = 1 asks a push partition for the staged scatter.
static bool stage_ok_push(const tc_part_params *pp) { return pp && pp->smem_stage > 0; }

// ---------------------------------------------------------------------------------------------
// Direct pieces.  Edge e of the blocked CSR alone forms its local row when it starts a row and
// the next edge starts one too; in the first Bd blocks (edges below e_cut) such pieces leave the
// CSR.  keep[e] = 0 marks them; keep[E] = 0 closes the scan.
// ---------------------------------------------------------------------------------------------
__global__ void k_direct_keep(const uint8_t *head, int64_t E, int64_t e_cut, int32_t *keep) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e <= E; e += (int64_t)gridDim.x * blockDim.x) {
        if (e == E) {
            keep[e] = 0;
            continue;
        }
        const bool single = head[e] && (e + 1 == E || head[e + 1]);
        keep[e] = (single && e < e_cut) ? 0 : 1;
    }
}

// Kept edges move to pos[e]; dropped edge e becomes direct piece e - pos[e] (target, source).
__global__ void k_direct_split(const int32_t *colidx, const int32_t *rows_sorted, const int32_t *keep,
                               const int32_t *pos, int64_t E, int32_t *colidx_new, int32_t *dv, int32_t *du) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        if (keep[e]) {
            colidx_new[pos[e]] = colidx[e];
        } else {
            const int64_t d = e - pos[e];
            dv[d] = rows_sorted[e];
            du[d] = colidx[e];
        }
    }
}

// rkeep[r] = whether local row r stays (its first edge is kept); rkeep[R] = 0.
__global__ void k_direct_rkeep(const int32_t *rowptr, int64_t R, const int32_t *keep, int32_t *rkeep) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= R; r += (int64_t)gridDim.x * blockDim.x)
        rkeep[r] = r < R ? keep[rowptr[r]] : 0;
}

__global__ void k_direct_rows(const int32_t *rowptr, const int32_t *id_map, int64_t R, const int32_t *rkeep,
                              const int32_t *rpos, const int32_t *pos, int32_t *rowptr_new, int32_t *id_map_new) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        if (!rkeep[r]) continue;
        const int32_t nr = rpos[r];
        rowptr_new[nr] = pos[rowptr[r]];
        id_map_new[nr] = id_map[r];
    }
}

// dir_off[j] = first direct piece whose target is >= rstart[j] (targets sorted); [nranges] = n.
__global__ void k_direct_off(const int32_t *dv, int64_t n, const int32_t *rstart, int32_t nranges, int32_t *dir_off) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= nranges; j += gridDim.x * blockDim.x) {
        if (j == nranges) {
            dir_off[j] = (int32_t)n;
            continue;
        }
        const int32_t want = rstart[j];
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (dv[mid] < want) lo = mid + 1; else hi = mid;
        }
        dir_off[j] = (int32_t)lo;
    }
}

// Take the single-edge pieces of the first Bd blocks out of the blocked CSR (rowptr, id_map,
// colidx, block bounds and their host copies are replaced) into the direct arrays, sorted by
// target and indexed per merge range (rstart).  head / rows_sorted describe the current CSR.
static int split_direct(tc_part *p, int32_t Bd, const uint8_t *head, const int32_t *rows_sorted,
                        const int32_t *rstart, DevBuf &blk_rows, DevBuf &blk_edges, cudaStream_t s, int grid) {
    const int64_t E = p->E, R = p->R;
    const int32_t B = p->B;
    const int64_t e_cut = p->h_blk_edges[Bd];
    DevBuf keep, pos;
    TC_TRY(keep.alloc(((size_t)E + 1) * 4));
    TC_TRY(pos.alloc(((size_t)E + 1) * 4));
    k_direct_keep<<<grid, 256, 0, s>>>(head, E, e_cut, keep.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32(keep.as<int32_t>(), E + 1, pos.as<int32_t>(), s));
    int32_t En = 0;
    TC_CUDA(cudaMemcpyAsync(&En, pos.as<int32_t>() + E, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    const int64_t Nd = E - En;
    p->Bd = Bd;
    p->ndirect = Nd;
    if (Nd == 0) return TC_OK;
    DevBuf col_new, dv, du;
    TC_TRY(col_new.alloc((size_t)(En > 0 ? En : 1) * 4));
    TC_TRY(dv.alloc((size_t)Nd * 4));
    TC_TRY(du.alloc((size_t)Nd * 4));
    k_direct_split<<<grid, 256, 0, s>>>(p->colidx.as<int32_t>(), rows_sorted, keep.as<int32_t>(), pos.as<int32_t>(), E,
                                        col_new.as<int32_t>(), dv.as<int32_t>(), du.as<int32_t>());
    TC_LAUNCH_CHECK();
    // rows
    DevBuf rkeep, rpos, rp_new, im_new;
    TC_TRY(rkeep.alloc(((size_t)R + 1) * 4));
    TC_TRY(rpos.alloc(((size_t)R + 1) * 4));
    k_direct_rkeep<<<grid, 256, 0, s>>>(p->rowptr.as<int32_t>(), R, keep.as<int32_t>(), rkeep.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32(rkeep.as<int32_t>(), R + 1, rpos.as<int32_t>(), s));
    int32_t Rn = 0;
    TC_CUDA(cudaMemcpyAsync(&Rn, rpos.as<int32_t>() + R, 4, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaStreamSynchronize(s));
    TC_TRY(rp_new.alloc(((size_t)Rn + 1) * 4));
    TC_TRY(im_new.alloc(((size_t)Rn + 8) * 4));
    TC_CUDA(cudaMemsetAsync(im_new.p, 0, ((size_t)Rn + 8) * 4, s));
    k_direct_rows<<<grid, 256, 0, s>>>(p->rowptr.as<int32_t>(), p->id_map.as<int32_t>(), R, rkeep.as<int32_t>(),
                                       rpos.as<int32_t>(), pos.as<int32_t>(), rp_new.as<int32_t>(), im_new.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaMemcpyAsync(rp_new.as<int32_t>() + Rn, &En, 4, cudaMemcpyHostToDevice, s));
    p->colidx.swap(col_new);
    p->rowptr.swap(rp_new);
    p->id_map.swap(im_new);
    p->E = En;
    p->R = Rn;
    k_block_bounds<<<(B + 256) / 256, 256, 0, s>>>(p->colidx.as<int32_t>(), p->rowptr.as<int32_t>(), En, Rn, p->W, B,
                                                   blk_edges.as<int64_t>(), blk_rows.as<int64_t>());
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaMemcpyAsync(p->h_blk_rows, blk_rows.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(p->h_blk_edges, blk_edges.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(p->blk_rows_dev.p, blk_rows.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToDevice, s));
    // the direct pieces by target (stable: block order within a target), then per merge range
    DevBuf dvs, dus, kt, vt;
    TC_TRY(dvs.alloc((size_t)Nd * 4));
    TC_TRY(p->dir_u.alloc(((size_t)Nd + 8) * 4));
    TC_TRY(kt.alloc((size_t)Nd * 4));
    TC_TRY(vt.alloc((size_t)Nd * 4));
    TC_CUDA(cudaMemsetAsync(p->dir_u.p, 0, ((size_t)Nd + 8) * 4, s));
    TC_TRY(stable_bucket_sort(dv.as<int32_t>(), du.as<int32_t>(), dvs.as<int32_t>(), p->dir_u.as<int32_t>(),
                              kt.as<int32_t>(), vt.as<int32_t>(), Nd, 1, log2_ceil(p->V > 1 ? p->V : 2), s));
    TC_TRY(p->dir_off.alloc(((size_t)p->nranges + 1) * 4));
    k_direct_off<<<(p->nranges + 256) / 256, 256, 0, s>>>(dvs.as<int32_t>(), Nd, rstart, p->nranges,
                                                          p->dir_off.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(p->dir_id16.alloc(((size_t)Nd + 8) * 2));
    TC_CUDA(cudaMemsetAsync(p->dir_id16.p, 0, ((size_t)Nd + 8) * 2, s));
    k_id16_ranges<<<grid, 256, 0, s>>>(dvs.as<int32_t>(), Nd, rstart, p->nranges, p->dir_id16.as<uint16_t>());
    TC_LAUNCH_CHECK();
    TC_CUDA(cudaStreamSynchronize(s));  // the scratch buffers are freed at return
    return TC_OK;
}

// Merge ranges that hold about equal work over the vertices [0, V') with V' = ni (the rest have
// no edge at all): vertex v weighs (pieces with destination v) + c, with c = max(1, ceil(R / V'));
// nr = ceil(2V' / (kmax - 64)) ranges split the total weight evenly, at multiples of 32.  As every
// vertex weighs at least c and R <= c V', no range is wider than kmax.
static int weighted_ranges(tc_part *p, int32_t kmax, cudaStream_t s, int grid) {
    const int32_t V = p->ni;  // the vertices from ni on have no edge: no range covers them
    const int64_t R = p->R;
    DevBuf cnt, cum;
    TC_TRY(cnt.alloc(((size_t)V + 1) * 4));
    TC_TRY(cum.alloc(((size_t)V + 1) * 8));
    TC_CUDA(cudaMemsetAsync(cnt.p, 0, ((size_t)V + 1) * 4, s));
    if (R > 0) {
        k_pieces_per_vertex<<<grid, 256, 0, s>>>(p->id_map.as<int32_t>(), R, cnt.as<int32_t>());
        TC_LAUNCH_CHECK();
    }
    const int32_t c = (int32_t)(R > V ? (R + V - 1) / V : 1);
    k_range_weights<<<grid, 256, 0, s>>>(cnt.as<int32_t>(), V, c);
    TC_LAUNCH_CHECK();
    TC_TRY(scan_i32_to_i64(cnt.as<int32_t>(), (int64_t)V + 1, cum.as<int64_t>(), s));
    const int64_t nr64 = ((int64_t)2 * V + (kmax - 64) - 1) / (kmax - 64);
    const int32_t nr = (int32_t)(nr64 > 0 ? nr64 : 1);
    TC_TRY(p->rstart.alloc(((size_t)nr + 1) * 4));
    k_range_bounds<<<(nr + 256) / 256, 256, 0, s>>>(cum.as<int64_t>(), V, nr, p->rstart.as<int32_t>());
    TC_LAUNCH_CHECK();
    // the width bound holds by construction; check it once on the host all the same
    int32_t *h = new (std::nothrow) int32_t[nr + 1];
    if (!h) return fail(TC_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, p->rstart.p, ((size_t)nr + 1) * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int32_t widest = 0;
    bool monotone = true;
    for (int32_t j = 0; e == cudaSuccess && j < nr; ++j) {
        const int32_t w = h[j + 1] - h[j];
        if (w < 0) monotone = false;
        if (w > widest) widest = w;
    }
    const bool ends_ok = e != cudaSuccess || (h[0] == 0 && h[nr] == V);
    delete[] h;
    if (e != cudaSuccess) return fail(TC_ERR_CUDA, "weighted_ranges: %s", cudaGetErrorString(e));
    if (!monotone || !ends_ok || widest > kmax)
        return fail(TC_ERR_CUDA, "weighted_ranges: internal error (widest range %d > %d)", widest, kmax);
    p->nranges = nr;
    return TC_OK;
}

static int partition_impl(const tc_graph *g, int dir, int32_t num_blocks, const tc_part_params *pp, cudaStream_t s,
                          tc_part *p) {
    DeviceCaps caps;
    TC_TRY(device_caps(&caps));
    const int32_t V = g->V;
    const int64_t E = g->E;
    const int32_t *rp = dir == TC_PULL ? g->in_rowptr.as<int32_t>() : g->out_rowptr.as<int32_t>();
    const int32_t *ci = dir == TC_PULL ? g->in_colidx.as<int32_t>() : g->out_colidx.as<int32_t>();
    p->g = g;
    p->dir = dir;
    p->V = V;
    p->E = E;
    const int order = pp ? pp->vertex_order : TC_ORDER_NATURAL;
    if (order != TC_ORDER_NATURAL && order != TC_ORDER_OUTDEGREE)
        return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: bad vertex_order");
    if (order == TC_ORDER_OUTDEGREE && dir != TC_PULL)
        return fail(TC_ERR_UNSUPPORTED, "tc_tocab_partition: push partitions cannot be renumbered");
    if (order == TC_ORDER_OUTDEGREE && pp && pp->merge_range > 0 && pp->merge_range < 128)
        return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: renumbered partitions need merge_range >= 128");
    DevBuf rel_rowptr, rel_colidx, rows_in;
    p->nz_out = (int32_t)((int64_t)V - g->num_dangling);  // vertices with out-edges
    p->ni = V;
    if (order == TC_ORDER_OUTDEGREE && V > 0) {
        TC_TRY(renumber_by_outdegree(g, s, &rel_rowptr, &rel_colidx, &rows_in, p));
        rp = rel_rowptr.as<int32_t>();
        ci = rel_colidx.as<int32_t>();
    }
    const float frac = (pp && pp->l2_fraction > 0) ? pp->l2_fraction : 0.0f;
    if (pp && pp->merge_range > 0) {
        p->k = pp->merge_range;
    } else {  // 8192 (longest slices that fit well), smaller for small graphs: >= 2 ranges per SM
        int64_t k = 8192;
        while (k > 1024 && ((int64_t)V + k - 1) / k < 2 * caps.sms) k >>= 1;
        p->k = (int32_t)k;
    }
    if (p->k % 32 != 0) return fail(TC_ERR_INVALID_ARG, "merge_range must be a multiple of 32");
    p->hub_degree = (pp && pp->hub_degree > 0) ? pp->hub_degree : 2048;
    const int32_t smem_w = tile_max_width(caps.max_smem_optin);
    const int policy = pp ? pp->block_policy : TC_BLOCKS_L2;
    if (num_blocks == 0 && policy == TC_BLOCKS_SMEM && dir == TC_PUSH) {
        // push: the widest destination range whose 8-byte sums fit one CTA's shared memory
        const int32_t pw = push_smem_width(caps.max_smem_optin);
        p->W = pw > 0 ? (V < pw ? (V > 32 ? (V + 31) / 32 * 32 : 32) : pw) : 32;
    } else if (num_blocks == 0 && policy == TC_BLOCKS_SMEM && p->order == TC_ORDER_OUTDEGREE) {
        // the gather splits blocks into row-aligned pieces of equal size, so B need not fill
        // whole waves: the widest block that fits shared memory gives the fewest pieces
        p->W = smem_w > 0 ? smem_w : 32;
    } else if (num_blocks == 0 && policy == TC_BLOCKS_SMEM) {
        // the smallest multiple of the SM count of blocks whose width fits shared memory:
        // one CTA per block, whole waves
        int64_t m = 1, Wc = 1;
        for (;; ++m) {
            Wc = ((int64_t)V + m * caps.sms - 1) / (m * caps.sms);
            Wc = (Wc + 31) / 32 * 32;
            if (Wc <= smem_w) break;
        }
        p->W = (int32_t)(Wc > 0 ? Wc : 32);
    } else if (num_blocks == 0) {
        p->W = tc_default_block_width(V, caps.l2_bytes, frac);
    } else {
        p->W = V > 0 ? (int32_t)(((int64_t)V + num_blocks - 1) / num_blocks) : 1;
        if (p->W > 32) p->W = (p->W + 31) / 32 * 32;  // 128-byte aligned source ranges
    }
    if (p->W < 1) p->W = 1;
    // renumbered: sources are exactly [0, nz_out), so the blocks past them would be empty
    const int64_t span = p->order == TC_ORDER_OUTDEGREE ? (int64_t)p->nz_out : (int64_t)V;
    p->B = span > 0 ? (int32_t)((span + p->W - 1) / p->W) : 1;
    p->nranges = (int32_t)(((int64_t)V + p->k - 1) / p->k);
    if (dir == TC_PULL && p->B > 65535)
        return fail(TC_ERR_UNSUPPORTED, "more than 65535 blocks");
    if (dir == TC_PULL && (int64_t)merge_atomic_smem_bytes(p->k, p->B, true) > (int64_t)caps.max_smem_optin)
        return fail(TC_ERR_INVALID_ARG, "merge_range %d with this block count needs more shared memory than a CTA has",
                    p->k);
    const int32_t B = p->B, W = p->W;
    const int grid = caps.sms * 8;

    TC_TRY(p->colidx.alloc((size_t)E * 4));
    DevBuf rows_sorted, head, head_prefix, ktmp, vtmp;
    TC_TRY(rows_sorted.alloc((size_t)E * 4));
    if (E > 0) {
        if (!rows_in.p) {  // (the renumbering has built it already)
            TC_TRY(rows_in.alloc((size_t)E * 4));
            TC_TRY(expand_rows(rp, V, rows_in.as<int32_t>(), s));
        }
        if (B > 1) {
            TC_TRY(ktmp.alloc((size_t)E * 4));
            TC_TRY(vtmp.alloc((size_t)E * 4));
            TC_TRY(stable_bucket_sort(ci, rows_in.as<int32_t>(), p->colidx.as<int32_t>(), rows_sorted.as<int32_t>(),
                                      ktmp.as<int32_t>(), vtmp.as<int32_t>(), E, W, log2_ceil(B), s));
            ktmp.release();
            vtmp.release();
        } else {
            TC_CUDA(cudaMemcpyAsync(p->colidx.p, ci, (size_t)E * 4, cudaMemcpyDeviceToDevice, s));
            TC_CUDA(cudaMemcpyAsync(rows_sorted.p, rows_in.p, (size_t)E * 4, cudaMemcpyDeviceToDevice, s));
        }
        rows_in.release();
        TC_TRY(head.alloc((size_t)E + 8));
        k_row_heads<<<grid, 256, 0, s>>>(p->colidx.as<int32_t>(), rows_sorted.as<int32_t>(), E, div_by(W),
                                          head.as<uint8_t>());
        TC_LAUNCH_CHECK();
        TC_TRY(head_tiles(head.as<uint8_t>(), E, &head_prefix, &p->R, s));
    } else {
        p->R = 0;
    }
    int64_t R = p->R;
    TC_TRY(p->rowptr.alloc(((size_t)R + 1) * 4));
    TC_TRY(p->id_map.alloc((size_t)(R + 8) * 4));  // padded: the merge reads whole 4-entry granules
    DevBuf blk_edges, blk_rows;
    TC_TRY(blk_edges.alloc(((size_t)B + 1) * 8));
    TC_TRY(blk_rows.alloc(((size_t)B + 1) * 8));
    if (E > 0) {
        TC_TRY(head_fill(head.as<uint8_t>(), E, head_prefix.as<int32_t>(), rows_sorted.as<int32_t>(),
                         p->rowptr.as<int32_t>(), p->id_map.as<int32_t>(), s));
        k_block_bounds<<<(B + 256) / 256, 256, 0, s>>>(p->colidx.as<int32_t>(), p->rowptr.as<int32_t>(), E, R, W, B,
                                                       blk_edges.as<int64_t>(), blk_rows.as<int64_t>());
        TC_LAUNCH_CHECK();
    } else {
        TC_CUDA(cudaMemsetAsync(blk_edges.p, 0, ((size_t)B + 1) * 8, s));
        TC_CUDA(cudaMemsetAsync(blk_rows.p, 0, ((size_t)B + 1) * 8, s));
    }
    const int32_t Ei = (int32_t)E;
    TC_CUDA(cudaMemcpyAsync(p->rowptr.as<int32_t>() + R, &Ei, 4, cudaMemcpyHostToDevice, s));
    p->h_blk_rows = new (std::nothrow) int64_t[B + 1];
    p->h_blk_edges = new (std::nothrow) int64_t[B + 1];
    if (!p->h_blk_rows || !p->h_blk_edges) return fail(TC_ERR_OOM, "host allocation failed");
    TC_CUDA(cudaMemcpyAsync(p->h_blk_rows, blk_rows.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, s));
    TC_CUDA(cudaMemcpyAsync(p->h_blk_edges, blk_edges.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, s));
    TC_TRY(p->blk_rows_dev.alloc(((size_t)B + 1) * 8));
    TC_CUDA(cudaMemcpyAsync(p->blk_rows_dev.p, blk_rows.p, ((size_t)B + 1) * 8, cudaMemcpyDeviceToDevice, s));

    // merge ranges: fixed width k, or (renumbered) cut to about equal work
    const int32_t *rst = nullptr;
    if (p->order == TC_ORDER_OUTDEGREE && V > 0) {
        TC_TRY(weighted_ranges(p, p->k, s, grid));
        rst = p->rstart.as<int32_t>();
    }
    // direct pieces (renumbered pull partitions; the ranges above still count them as pieces,
    // which they remain for the merge)
    if (rst && dir == TC_PULL && E > 0 && R > 0 && pp && pp->direct_blocks != 0) {
        int64_t bd = pp->direct_blocks > 0 ? (int64_t)pp->direct_blocks
                                           : (int64_t)(caps.l2_bytes / 8) / ((int64_t)W * 4);
        if (bd < 1) bd = 1;
        if (bd > B) bd = B;
        TC_TRY(split_direct(p, (int32_t)bd, head.as<uint8_t>(), rows_sorted.as<int32_t>(), rst, blk_rows, blk_edges, s,
                            grid));
        R = p->R;
    }
    // merge range table
    const int64_t noff = (int64_t)B * (p->nranges + 1);
    TC_TRY(p->merge_off.alloc((size_t)(noff > 0 ? noff : 1) * 4));
    TC_TRY(p->merge_offT.alloc((size_t)(noff > 0 ? noff : 1) * 4));
    if (noff > 0) {
        k_merge_offsets<<<grid, 256, 0, s>>>(p->id_map.as<int32_t>(), blk_rows.as<int64_t>(), B, p->nranges, p->k,
                                             rst, p->merge_off.as<int32_t>(), p->merge_offT.as<int32_t>());
        TC_LAUNCH_CHECK();
    }
    TC_TRY(p->merge_gpre.alloc((size_t)p->nranges * ((size_t)B + 1) * 4));
    k_merge_gpre<<<grid, 256, 0, s>>>(p->merge_offT.as<int32_t>(), B, p->nranges, p->merge_gpre.as<int32_t>());
    TC_LAUNCH_CHECK();
    TC_TRY(collect_hubs(p->rowptr.as<int32_t>(), R, p->hub_degree, &p->hubs, &p->num_hubs, s));
    if (R > 0 && rst) {  // 2-byte offsets inside the (variable) merge ranges, all <= k <= 65536
        TC_TRY(p->id16.alloc((size_t)(R + 8) * 2));
        k_id16_ranges<<<grid, 256, 0, s>>>(p->id_map.as<int32_t>(), R, rst, p->nranges, p->id16.as<uint16_t>());
        TC_LAUNCH_CHECK();
    } else if (R > 0 && (p->k & (p->k - 1)) == 0 && p->k <= 65536) {  // 2-byte local ids for the merge
        TC_TRY(p->id16.alloc((size_t)(R + 8) * 2));
        k_id16<<<grid, 256, 0, s>>>(p->id_map.as<int32_t>(), R, p->k - 1, p->id16.as<uint16_t>());
        TC_LAUNCH_CHECK();
    }
    // push: the source of every edge in stream order (the sort's row values), for the
    // edge-parallel scatter
    if (dir == TC_PUSH) p->esrc.swap(rows_sorted);
    // push ranges that fit shared memory get the staged scatter (tc_push.cu)
    if (dir == TC_PUSH && (int64_t)W * 8 + 1024 <= (int64_t)caps.max_smem_optin && stage_ok_push(pp))
        TC_TRY(build_push_tiles(p, caps.sms, s));
    p->num_groups = (R + 31) / 32;
    TC_TRY(p->partial.alloc((size_t)(R + 8) * 4));
    TC_TRY(p->rowbits.alloc((size_t)((R + 31) / 32 + 1) * 4));
    TC_CUDA(cudaStreamSynchronize(s));
    const int stage = pp ? pp->smem_stage : 0;
    if (stage > 0 && dir == TC_PUSH && p->nptiles == 0 && E > 0)
        return fail(TC_ERR_UNSUPPORTED, "smem_stage = 1 needs a push partition with W * 8 bytes within shared memory");
    if (dir == TC_PULL && stage >= 0 && W <= smem_w && W % 32 == 0 && V > 0)
        TC_TRY(build_tiles(p, caps.sms, s));
    if (stage > 0 && dir == TC_PULL && !p->tiled)
        return fail(TC_ERR_UNSUPPORTED, "smem_stage = 1 needs a pull partition with W <= %d and W %% 32 == 0", smem_w);
    return TC_OK;
}

}  // namespace tc

extern "C" int32_t tc_default_block_width(int32_t V, int64_t l2_bytes, float l2_fraction) {
    // Default: the paper's 256 Ki FP32 values on a 2.75 MB (= 11 x 256 KiB) L2, i.e. the
    // block's vertex values take 4/11 of the L2 and W = l2_bytes / 11 exactly.
    int64_t W = l2_fraction > 0 ? (int64_t)((double)l2_fraction * (double)l2_bytes / 4.0) : l2_bytes / 11;
    if (W < 32) W = 32;
    if (V > 0 && W > V) W = V;
    if (W > INT32_MAX) W = INT32_MAX;
    return (int32_t)W;
}

extern "C" int tc_tocab_partition(const tc_graph *g, int dir, int32_t num_blocks, const tc_part_params *params,
                                  void *stream, tc_part **out) {
    using namespace tc;
    if (!out) return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: out is NULL");
    *out = nullptr;
    if (!g) return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: graph is NULL");
    if (dir != TC_PULL && dir != TC_PUSH) return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: bad direction");
    if (num_blocks < 0 || (g->V > 0 && num_blocks > g->V))
        return fail(TC_ERR_INVALID_ARG, "tc_tocab_partition: num_blocks must be in [0, V]");
    tc_part *p = new (std::nothrow) tc_part();
    if (!p) return fail(TC_ERR_OOM, "host allocation failed");
    int st = partition_impl(g, dir, num_blocks, params, (cudaStream_t)stream, p);
    if (st != TC_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        delete p;
        return st;
    }
    *out = p;
    return TC_OK;
}

extern "C" void tc_part_free(tc_part *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
}

extern "C" int tc_part_get_info(const tc_part *p, tc_part_info *info) {
    if (!p || !info) return tc::fail(TC_ERR_INVALID_ARG, "tc_part_get_info: null argument");
    info->dir = p->dir;
    info->num_blocks = p->B;
    info->block_width = p->W;
    info->num_rows = p->R;
    info->num_edges = p->E;
    info->merge_range = p->k;
    info->num_hubs = p->num_hubs;
    info->staged = p->tiled ? 1 : 0;
    info->staged_edges = p->padded_edges;
    info->vertex_order = p->order;
    info->num_ranges = p->nranges;
    info->num_tiles = p->tiled ? p->ntiles : 0;
    info->num_sources = p->nz_out;
    info->direct_blocks = p->Bd;
    info->num_direct = p->ndirect;
    return TC_OK;
}

extern "C" int tc_part_export_order(const tc_part *p, int32_t *perm, int mem, void *stream) {
    using namespace tc;
    if (!p || !perm) return fail(TC_ERR_INVALID_ARG, "tc_part_export_order: null argument");
    if (mem != TC_MEM_HOST && mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "bad mem flag");
    cudaStream_t s = (cudaStream_t)stream;
    if (p->V == 0) return TC_OK;
    if (p->order == TC_ORDER_OUTDEGREE) {
        TC_CUDA(cudaMemcpyAsync(perm, p->perm.p, (size_t)p->V * 4,
                                mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
        TC_CUDA(cudaStreamSynchronize(s));
        return TC_OK;
    }
    if (mem == TC_MEM_HOST) {
        for (int32_t n = 0; n < p->V; ++n) perm[n] = n;
        return TC_OK;
    }
    int32_t *h = new (std::nothrow) int32_t[p->V];
    if (!h) return fail(TC_ERR_OOM, "host allocation failed");
    for (int32_t n = 0; n < p->V; ++n) h[n] = n;
    cudaError_t e = cudaMemcpyAsync(perm, h, (size_t)p->V * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    delete[] h;
    if (e != cudaSuccess) return fail(TC_ERR_CUDA, "tc_part_export_order: %s", cudaGetErrorString(e));
    return TC_OK;
}

extern "C" int tc_part_export(const tc_part *p, int64_t *blk_rows, int64_t *blk_edges, int32_t *rowptr,
                              int32_t *id_map, int32_t *colidx, int mem, void *stream) {
    using namespace tc;
    if (!p) return fail(TC_ERR_INVALID_ARG, "tc_part_export: null partition");
    if (mem != TC_MEM_HOST && mem != TC_MEM_DEVICE) return fail(TC_ERR_INVALID_ARG, "bad mem flag");
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind d2x = mem == TC_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const cudaMemcpyKind h2x = mem == TC_MEM_DEVICE ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    if (blk_rows) TC_CUDA(cudaMemcpyAsync(blk_rows, p->h_blk_rows, ((size_t)p->B + 1) * 8, h2x, s));
    if (blk_edges) TC_CUDA(cudaMemcpyAsync(blk_edges, p->h_blk_edges, ((size_t)p->B + 1) * 8, h2x, s));
    if (rowptr) TC_CUDA(cudaMemcpyAsync(rowptr, p->rowptr.p, ((size_t)p->R + 1) * 4, d2x, s));
    if (id_map && p->R > 0) TC_CUDA(cudaMemcpyAsync(id_map, p->id_map.p, (size_t)p->R * 4, d2x, s));
    if (colidx && p->E > 0) TC_CUDA(cudaMemcpyAsync(colidx, p->colidx.p, (size_t)p->E * 4, d2x, s));
    TC_CUDA(cudaStreamSynchronize(s));
    return TC_OK;
}

extern "C" int tc_part_set_lb(tc_part *p, const int32_t *warp_min_per_block) {
    using namespace tc;
    if (!p) return fail(TC_ERR_INVALID_ARG, "tc_part_set_lb: null partition");
    if (!warp_min_per_block) {
        p->lb_tab.release();
        return TC_OK;
    }
    for (int32_t b = 0; b < p->B; ++b)
        if (warp_min_per_block[b] < 1) return fail(TC_ERR_INVALID_ARG, "tc_part_set_lb: warp_min must be >= 1");
    TC_TRY(p->lb_tab.alloc((size_t)p->B * 4));
    TC_CUDA(cudaMemcpy(p->lb_tab.p, warp_min_per_block, (size_t)p->B * 4, cudaMemcpyHostToDevice));
    return TC_OK;
}
