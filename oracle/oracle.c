/*
 * Plain, slow, obviously-correct FP64 CPU oracle for the TOCAB hot path of
 * "GraphCage: Cache Aware Graph Processing on GPUs" (Chen, 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the GPU library includes, links or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header or table with the CUDA path.
 *
 * Every function follows the definition in the cited section of the paper, with no
 * blocking, fusion or reordering beyond what that definition states.  Where the paper
 * is silent (dangling vertices, initial ranks, personalised teleport), the reading
 * taken is named in the comment.
 *
 * Graphs: CSR with int32 row offsets (rowptr[V+1]) and int32 column indices.
 * "out-CSR" = rows are sources, columns destinations (the graph G);
 * "in-CSR"  = rows are destinations, columns sources (the transpose G^T).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-3)

/* ------------------------------------------------------------------------------------
 * Transpose: G (out-CSR) -> G^T (in-CSR).  Sec. 2.1 (CSR), Alg. 1 reads G^T.
 * Counting sort by destination; sources are visited in ascending order, so every
 * in-row comes out sorted by source id.
 * ---------------------------------------------------------------------------------- */
int orc_transpose(int32_t V, int64_t E, const int32_t *rowptr, const int32_t *colidx,
                  int32_t *t_rowptr, int32_t *t_colidx)
{
    if (V < 0 || E < 0) return ORC_EINVAL;
    int64_t *cursor = (int64_t *)calloc((size_t)V + 1, sizeof(int64_t));
    if (!cursor) return ORC_ENOMEM;
    for (int64_t e = 0; e < E; ++e) cursor[colidx[e] + 1] += 1;       /* in-degree */
    for (int32_t v = 0; v < V; ++v) cursor[v + 1] += cursor[v];        /* offsets   */
    for (int32_t v = 0; v <= V; ++v) t_rowptr[v] = (int32_t)cursor[v];
    for (int32_t u = 0; u < V; ++u)
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t v = colidx[e];
            t_colidx[cursor[v]++] = u;
        }
    free(cursor);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Pull PageRank, Alg. 1 (Sec. 2.2), FP64, Jacobi iterations.
 *   contributions[u] = rank[u] / out_degree[u]            (0 when out_degree[u] == 0)
 *   sums[v]          = sum over in-neighbours u of contributions[u]
 *   rank[v]          = (1-d)/|V| + d * (sums[v] + D/|V|)
 * D is the rank mass on dangling vertices (out_degree 0); with dangling_mode == 1
 * ("drop") the D/|V| term is omitted, which is Alg. 1 read literally (mass leaks).
 * Initial rank: 1/|V| everywhere unless init != NULL.
 * nthreads > 1 parallelises the destination loop only; every sums[v] is still
 * accumulated serially in in-row order, so the result does not depend on nthreads.
 * ---------------------------------------------------------------------------------- */
int orc_pagerank_pull(int32_t V, const int32_t *in_rowptr, const int32_t *in_colidx,
                      const int32_t *out_degree, double damping, int32_t iters,
                      int32_t dangling_mode, const double *init, double *rank, int32_t nthreads)
{
    if (V <= 0 || iters < 0) return ORC_EINVAL;
    double *contrib = (double *)malloc((size_t)V * sizeof(double));
    if (!contrib) return ORC_ENOMEM;
    for (int32_t v = 0; v < V; ++v) rank[v] = init ? init[v] : 1.0 / (double)V;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int32_t it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (int32_t u = 0; u < V; ++u) {                 /* Alg. 1: contributions   */
            if (out_degree[u] > 0) contrib[u] = rank[u] / (double)out_degree[u];
            else { contrib[u] = 0.0; dangling += rank[u]; }
        }
        double base = (1.0 - damping) / (double)V;
        double spread = (dangling_mode == 0) ? dangling / (double)V : 0.0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4096) if (nthreads > 1)
#endif
        for (int32_t v = 0; v < V; ++v) {                 /* Alg. 1: in-edge sums    */
            double sum = 0.0;
            for (int64_t e = in_rowptr[v]; e < in_rowptr[v + 1]; ++e) sum += contrib[in_colidx[e]];
            rank[v] = base + damping * (sum + spread);    /* Alg. 1: rank update     */
        }
    }
    free(contrib);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Push PageRank, Alg. 2 (Sec. 2.2), FP64: scatter every contribution along out-edges
 * of G into sums, then the same update as Alg. 1.  Same readings for dangling mass and
 * initial ranks.  Serial (the atomics of Alg. 2 are only needed in parallel).
 * ---------------------------------------------------------------------------------- */
int orc_pagerank_push(int32_t V, const int32_t *rowptr, const int32_t *colidx,
                      double damping, int32_t iters, int32_t dangling_mode,
                      const double *init, double *rank)
{
    if (V <= 0 || iters < 0) return ORC_EINVAL;
    double *sums = (double *)malloc((size_t)V * sizeof(double));
    if (!sums) return ORC_ENOMEM;
    for (int32_t v = 0; v < V; ++v) rank[v] = init ? init[v] : 1.0 / (double)V;
    for (int32_t it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (int32_t v = 0; v < V; ++v) sums[v] = 0.0;
        for (int32_t src = 0; src < V; ++src) {
            int64_t deg = (int64_t)rowptr[src + 1] - rowptr[src];
            if (deg == 0) { dangling += rank[src]; continue; }
            double c = rank[src] / (double)deg;           /* Alg. 2: contribution */
            for (int64_t e = rowptr[src]; e < rowptr[src + 1]; ++e)
                sums[colidx[e]] += c;                     /* Alg. 2: scatter      */
        }
        double base = (1.0 - damping) / (double)V;
        double spread = (dangling_mode == 0) ? dangling / (double)V : 0.0;
        for (int32_t v = 0; v < V; ++v) rank[v] = base + damping * (sums[v] + spread);
    }
    free(sums);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Personalised PageRank for a batch of sources, FP64 (pull form of Alg. 1 per column).
 * Readings: column j teleports to its source s_j, i.e. (1-d) e_{s_j}; the dangling mass
 * of column j also goes to s_j; the initial column is e_{s_j}.  R is V x n row-major
 * (R[v*n + j]).
 * ---------------------------------------------------------------------------------- */
int orc_ppr_pull(int32_t V, const int32_t *in_rowptr, const int32_t *in_colidx,
                 const int32_t *out_degree, double damping, int32_t iters,
                 int32_t n, const int32_t *srcs, double *R)
{
    if (V <= 0 || n <= 0 || iters < 0) return ORC_EINVAL;
    double *rank = (double *)malloc((size_t)V * sizeof(double));
    double *contrib = (double *)malloc((size_t)V * sizeof(double));
    if (!rank || !contrib) { free(rank); free(contrib); return ORC_ENOMEM; }
    for (int32_t j = 0; j < n; ++j) {
        int32_t s = srcs[j];
        if (s < 0 || s >= V) { free(rank); free(contrib); return ORC_EINVAL; }
        for (int32_t v = 0; v < V; ++v) rank[v] = (v == s) ? 1.0 : 0.0;
        for (int32_t it = 0; it < iters; ++it) {
            double dangling = 0.0;
            for (int32_t u = 0; u < V; ++u) {
                if (out_degree[u] > 0) contrib[u] = rank[u] / (double)out_degree[u];
                else { contrib[u] = 0.0; dangling += rank[u]; }
            }
            for (int32_t v = 0; v < V; ++v) {
                double sum = 0.0;
                for (int64_t e = in_rowptr[v]; e < in_rowptr[v + 1]; ++e) sum += contrib[in_colidx[e]];
                rank[v] = damping * sum + ((v == s) ? (1.0 - damping) + damping * dangling : 0.0);
            }
        }
        for (int32_t v = 0; v < V; ++v) R[(int64_t)v * n + j] = rank[v];
    }
    free(rank); free(contrib);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Level-synchronous BFS (Sec. 2.1 / Sec. 3.3 status arrays), over out-edges of G.
 * levels[s] = 0; a vertex first reached while expanding level L gets L+1;
 * unreachable vertices get -1 (the paper's "infinity", Alg. 3).
 * Textbook FIFO-queue BFS: the level of a vertex is its hop distance from s.
 * ---------------------------------------------------------------------------------- */
int orc_bfs(int32_t V, const int32_t *rowptr, const int32_t *colidx, int32_t source,
            int32_t *levels)
{
    if (V <= 0 || source < 0 || source >= V) return ORC_EINVAL;
    int32_t *queue = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    if (!queue) return ORC_ENOMEM;
    for (int32_t v = 0; v < V; ++v) levels[v] = -1;
    int64_t head = 0, tail = 0;
    levels[source] = 0;
    queue[tail++] = source;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {
            int32_t v = colidx[e];
            if (levels[v] < 0) { levels[v] = levels[u] + 1; queue[tail++] = v; }
        }
    }
    free(queue);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * TOCAB static 1D blocking, Sec. 3.1 (blocked CSR, Fig. 3; local IDs, Fig. 4).
 * Input: a CSR whose rows are the "output" vertices and whose columns are the
 * "input" vertices (for pull: G^T, rows = destinations, columns = sources; for push:
 * G, rows = sources, columns = destinations -- the same code, Sec. 3.1).
 * Block b holds every edge whose column lies in [b*W, min((b+1)*W, V)).
 * Within block b, only rows with at least one edge get a local ID; local IDs are given
 * in ascending order of the row's global ID (reading: the paper leaves the order open).
 * Outputs (all concatenated in block order):
 *   blk_rows[B+1]  : first local row of each block in the concatenated row space
 *   blk_edges[B+1] : first edge of each block
 *   rowptr[R+1]    : edge offsets of every local row (global positions), R = total rows
 *   id_map[R]      : global ID of every local row
 *   colidx[E]      : column (global) of every edge, in row order, columns ascending as
 *                    in the input row
 * Call with rowptr == NULL to get only blk_rows / blk_edges (sizes).
 * ---------------------------------------------------------------------------------- */
int orc_partition(int32_t V, const int32_t *in_rowptr, const int32_t *in_colidx,
                  int32_t W, int32_t B,
                  int64_t *blk_rows, int64_t *blk_edges,
                  int64_t *rowptr, int32_t *id_map, int32_t *colidx)
{
    if (V < 0 || W <= 0 || B <= 0 || (int64_t)B * W < V) return ORC_EINVAL;
    int64_t r = 0, e = 0;
    for (int32_t b = 0; b < B; ++b) {
        int64_t lo = (int64_t)b * W, hi = lo + W;
        blk_rows[b] = r;
        blk_edges[b] = e;
        for (int32_t v = 0; v < V; ++v) {
            int64_t cnt = 0;
            for (int64_t k = in_rowptr[v]; k < in_rowptr[v + 1]; ++k) {
                int32_t u = in_colidx[k];
                if (u >= lo && u < hi) {
                    if (rowptr) colidx[e + cnt] = u;
                    ++cnt;
                }
            }
            if (cnt > 0) {
                if (rowptr) { rowptr[r] = e; id_map[r] = v; }
                ++r;
                e += cnt;
            }
        }
    }
    blk_rows[B] = r;
    blk_edges[B] = e;
    if (rowptr) rowptr[r] = e;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Betweenness centrality, forward sweep: Alg. 3 (shortest-path calculation), over the
 * out-edges of G from one source s.  In the paper's notation delta is the depth and
 * sigma the number of shortest paths: delta[s] = 0, sigma[s] = 1; a vertex first reached
 * from a vertex of depth L gets depth L+1, and every edge src -> dst with
 * delta[dst] = delta[src] + 1 adds sigma[src] to sigma[dst].  Unreached vertices keep
 * depth -1 (the paper's infinity) and sigma 0.  Sigma is held in FP64 (exact below 2^53).
 * A FIFO queue visits vertices in nondecreasing depth, so sigma[src] is final when src is
 * expanded.  order[] receives the visiting order (its first *count entries).
 * ---------------------------------------------------------------------------------- */
int orc_bc_forward(int32_t V, const int32_t *rowptr, const int32_t *colidx, int32_t source,
                   int32_t *depth, double *sigma, int32_t *order, int32_t *count)
{
    if (V <= 0 || source < 0 || source >= V) return ORC_EINVAL;
    for (int32_t v = 0; v < V; ++v) { depth[v] = -1; sigma[v] = 0.0; }
    int64_t head = 0, tail = 0;
    depth[source] = 0;
    sigma[source] = 1.0;
    order[tail++] = source;
    while (head < tail) {
        int32_t src = order[head++];
        for (int64_t e = rowptr[src]; e < rowptr[src + 1]; ++e) {
            int32_t dst = colidx[e];
            if (depth[dst] < 0) { depth[dst] = depth[src] + 1; order[tail++] = dst; }
            if (depth[dst] == depth[src] + 1) sigma[dst] += sigma[src];
        }
    }
    *count = (int32_t)tail;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Betweenness centrality scores from a set of sources: for each source, Alg. 3's forward
 * sweep, then the backward sweep of the dependency accumulation the paper's BC reference
 * uses: visiting vertices in reverse forward order,
 *   dep[v] = sum over out-neighbours w of v with depth[w] = depth[v] + 1 of
 *            sigma[v] / sigma[w] * (1 + dep[w]),
 * and every vertex other than the source adds dep[v] to its score.  Reading: scores are the
 * plain sum over the given sources and over ordered targets (no normalisation, no halving
 * for undirected graphs).
 * ---------------------------------------------------------------------------------- */
int orc_bc(int32_t V, const int32_t *rowptr, const int32_t *colidx, int32_t nsrc,
           const int32_t *sources, double *score)
{
    if (V <= 0 || nsrc < 0) return ORC_EINVAL;
    int32_t *depth = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    int32_t *order = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    double *sigma = (double *)malloc((size_t)V * sizeof(double));
    double *dep = (double *)malloc((size_t)V * sizeof(double));
    if (!depth || !order || !sigma || !dep) {
        free(depth); free(order); free(sigma); free(dep);
        return ORC_ENOMEM;
    }
    for (int32_t v = 0; v < V; ++v) score[v] = 0.0;
    int rc = ORC_OK;
    for (int32_t k = 0; k < nsrc && rc == ORC_OK; ++k) {
        int32_t count = 0;
        rc = orc_bc_forward(V, rowptr, colidx, sources[k], depth, sigma, order, &count);
        if (rc != ORC_OK) break;
        for (int32_t v = 0; v < V; ++v) dep[v] = 0.0;
        for (int32_t i = count - 1; i >= 0; --i) {
            int32_t v = order[i];
            for (int64_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                int32_t w = colidx[e];
                if (depth[w] == depth[v] + 1) dep[v] += sigma[v] / sigma[w] * (1.0 + dep[w]);
            }
            if (v != sources[k]) score[v] += dep[v];
        }
    }
    free(depth); free(order); free(sigma); free(dep);
    return rc;
}

/* ------------------------------------------------------------------------------------
 * Sparse matrix-vector product y = A x (Sec. 4: SpMV as the generalised form of the graph
 * operators), with A in CSR: row i holds the entries A[i][colidx[k]] = vals[k] for
 * k in [rowptr[i], rowptr[i+1]).  Each y[i] is the sum of its row's products in the
 * row's storage order, in FP64.  In graph terms this is the pull gather of Alg. 1 with a
 * value on every edge (rows = destinations, columns = sources).
 * ---------------------------------------------------------------------------------- */
int orc_spmv(int32_t nrows, const int32_t *rowptr, const int32_t *colidx, const double *vals,
             const double *x, double *y)
{
    if (nrows < 0) return ORC_EINVAL;
    for (int32_t i = 0; i < nrows; ++i) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) acc += vals[k] * x[colidx[k]];
        y[i] = acc;
    }
    return ORC_OK;
}
