/*
 * tocab.h -- C ABI of the GB300 (sm_103a) throughput-oriented cache blocking (TOCAB)
 * library: pull/push PageRank and topology-driven pull BFS over CSR graphs, after
 * "GraphCage: Cache Aware Graph Processing on GPUs" (Chen, 2019).
 *
 * Conventions for every entry point
 *   - Return value: TC_OK (0) on success, a negative TC_ERR_* code otherwise; no
 *     exception or longjmp crosses this boundary.  On failure the outputs are
 *     unspecified and tc_last_error() returns a message for the calling thread.
 *   - Pointers are plain host or device addresses; where an argument can be either,
 *     a TC_MEM_HOST / TC_MEM_DEVICE flag says which.  Device pointers must belong to
 *     the device that is current when the call is made.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     All device work of a call is ordered on that stream; calls that return host data
 *     synchronise it.
 *   - The caller owns every input and output buffer.  Handles (tc_graph, tc_part) and
 *     their device scratch are owned by the library and released by the *_free calls.
 *     A handle may be used by one call at a time (calls on one handle must not overlap).
 *   - Vertex IDs and edge offsets are int32: V < 2^31 and E < 2^31, else
 *     TC_ERR_UNSUPPORTED.
 */
#ifndef TOCAB_H
#define TOCAB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------- */
#define TC_OK                  0
#define TC_ERR_INVALID_ARG    (-1)   /* bad pointer, size, flag or parameter            */
#define TC_ERR_INVALID_GRAPH  (-2)   /* CSR not monotone, column out of range, ...       */
#define TC_ERR_OOM            (-3)   /* device or host allocation failed                 */
#define TC_ERR_CUDA           (-4)   /* a CUDA runtime call failed (text in last error)  */
#define TC_ERR_TIMEOUT        (-5)   /* a bounded device-side wait gave up               */
#define TC_ERR_UNSUPPORTED    (-6)   /* size beyond int32 limits or unsupported option   */

/* ---- flags --------------------------------------------------------------------------- */
#define TC_MEM_HOST     0
#define TC_MEM_DEVICE   1

#define TC_PULL         0            /* blocks = source ranges of G^T (column blocking)  */
#define TC_PUSH         1            /* blocks = destination ranges of G (row blocking)   */

#define TC_DANGLING_REDISTRIBUTE 0   /* dangling rank mass spread uniformly (sum = 1)     */
#define TC_DANGLING_DROP         1   /* Alg. 1 read literally: dangling mass is dropped   */

typedef struct tc_graph tc_graph;    /* opaque: a graph resident on one device           */
typedef struct tc_part  tc_part;     /* opaque: a TOCAB partition of a tc_graph           */

/* ---- status ---------------------------------------------------------------------------- */
/* Static text for a status code (library utility, no counterpart in the paper; never fails). */
const char *tc_status_string(int status);
/* Message of the last failed call on this thread, "" if none (library utility, no counterpart
 * in the paper; the string is owned by the library and valid until the thread's next call). */
const char *tc_last_error(void);
/* Library version as 10000*major + 100*minor + patch (no counterpart in the paper). */
int tc_version(void);

/* ---- device memory budget ---------------------------------------------------------------- */
/*
 * tc_set_device_memory_limit -- caps the device memory the library holds at once (graphs,
 * partitions, workspaces and temporaries, on all devices together; blocks kept by its
 * allocation cache count as held; setting a cap returns the cached ones to the driver).
 * bytes = 0 removes the cap (the default).  An allocation
 * that would exceed the cap fails with TC_ERR_OOM and a message naming the cap; nothing
 * already allocated is freed.  tc_device_memory_held reports the bytes held now.  The paper
 * has no counterpart: this is for processes that share the GPU with other users of its
 * memory, and for testing the out-of-memory paths without exhausting the device.
 */
int tc_set_device_memory_limit(int64_t bytes);
int64_t tc_device_memory_held(void);

/* ---- graph ----------------------------------------------------------------------------- */
/*
 * tc_graph_load_csr -- copy a directed graph G = (V, E) given as an out-edge CSR
 * (rowptr int32[V+1], colidx int32[E]; row u lists the destinations of u's out-edges)
 * onto the current device, validate it, and build on the device the transpose G^T
 * (in-edge CSR, in-rows sorted by source) and the per-vertex out-degree reciprocals.
 * Sec. 2.1 (CSR, Fig. 1b); Alg. 1 pulls over G^T, Alg. 2 pushes over G.
 *   rowptr/colidx : host or device arrays per `mem`; not retained after the call.
 *   E             : must equal rowptr[V]; duplicates and self loops are kept as given.
 *   out           : receives the new handle (free with tc_graph_free).
 * Errors: TC_ERR_INVALID_ARG (null pointer, V < 0, E < 0), TC_ERR_INVALID_GRAPH
 * (rowptr[0] != 0, rowptr not monotone, rowptr[V] != E, colidx outside [0, V)),
 * TC_ERR_UNSUPPORTED (V or E >= 2^31), TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_graph_load_csr(int32_t V, int64_t E, const int32_t *rowptr, const int32_t *colidx,
                      int mem, void *stream, tc_graph **out);
/* Release a graph and its device memory; NULL is ignored (handle management, no counterpart in
 * the paper).  Waits for the device before freeing. */
void tc_graph_free(tc_graph *g);

typedef struct tc_graph_info {
    int32_t V;
    int64_t E;
    int32_t max_in_degree;
    int32_t max_out_degree;
    int64_t num_dangling;     /* vertices with out-degree 0 */
    int32_t device;
} tc_graph_info;
/* Sizes and degree statistics of a loaded graph: V and E of Sec. 2.1, and the dangling vertices
 * (out-degree 0) whose contribution step in Alg. 1 divides by zero.  Errors: TC_ERR_INVALID_ARG
 * for a NULL argument. */
int tc_graph_get_info(const tc_graph *g, tc_graph_info *info);

/*
 * tc_graph_export_transpose -- copy the device-built G^T that Alg. 1 pulls over (Sec. 2.1 CSR;
 * rowptr[V+1], colidx[E], in-rows sorted by source id) to caller-owned host or device buffers per
 * `mem`.  Synchronises.  Errors: TC_ERR_INVALID_ARG (NULL graph, bad mem), TC_ERR_CUDA.
 */
int tc_graph_export_transpose(const tc_graph *g, int32_t *rowptr, int32_t *colidx, int mem,
                              void *stream);

/* ---- TOCAB partition --------------------------------------------------------------------- */
/*
 * Sec. 3.1 "Throughput Oriented Cache Blocking", preprocessing phase: static 1D blocking.
 * TC_PULL: every edge of G^T goes to the block of its SOURCE, blocks are source ranges
 * [b*W, (b+1)*W) (column blocking; Fig. 3).  TC_PUSH: every edge of G goes to the block
 * of its DESTINATION (row blocking, the same code on the transposed input).
 * Inside a block only vertices with at least one edge get a local ID (Fig. 4), given in
 * ascending global-ID order; id_map maps local to global IDs.  All blocks are
 * concatenated in block order into one row space of R local rows.
 *   num_blocks : B >= 1 (W = ceil(V/B), rounded up to a multiple of 32 when above 32; the
 *                partition then has ceil(V/W) <= B blocks),
 *                or 0 to derive W from the device's L2 size: W FP32 vertex values take
 *                `l2_fraction` of cudaDeviceProp::l2CacheSize; the default (<= 0) is 4/11,
 *                i.e. W = l2CacheSize / 11 -- the paper's 256 Ki vertices per subgraph
 *                on its 2.75 MB L2 (Sec. 4.3, Table 3).
 * Errors: TC_ERR_INVALID_ARG (dir, B < 0, B > V when V > 0), TC_ERR_OOM, TC_ERR_CUDA.
 */
#define TC_BLOCKS_L2    0            /* num_blocks == 0: W from the L2 size (the paper's rule) */
#define TC_BLOCKS_SMEM  1            /* num_blocks == 0: W from one CTA's shared memory, B a
                                        multiple of the SM count (whole waves of CTAs)         */

typedef struct tc_part_params {
    float   l2_fraction;      /* used when num_blocks == 0 with TC_BLOCKS_L2; <= 0 means 4/11 */
    int32_t merge_range;      /* k of the merge (Fig. 5): vertices per merge CTA, a multiple of
                                 32; 0 = 8192 (halved down to 1024 while there would be
                                 fewer than two ranges per SM) */
    int32_t hub_degree;       /* rows with more edges go to CTA-per-row tasks; 0 = 2048 */
    int32_t block_policy;     /* TC_BLOCKS_L2 or TC_BLOCKS_SMEM (used when num_blocks == 0) */
    int32_t smem_stage;       /* pull: 0 = stage each block's contributions in shared
                                 memory whenever W fits (W <= about 41K sources, W % 32 == 0),
                                 -1 = never, 1 = require it (TC_ERR_UNSUPPORTED if W does not fit).
                                 push: 1 = accumulate each block's destination range in shared
                                 memory when W * 8 bytes fit (about 29K vertices; the
                                 TC_BLOCKS_SMEM policy picks that width), 0 / -1 = the global
                                 scatters.  Measured slower on R-MAT (shared-memory atomics on
                                 the hub destinations of a range serialise), so not the default */
    int32_t vertex_order;     /* pull only: TC_ORDER_NATURAL (0) or TC_ORDER_OUTDEGREE (1), below */
    int32_t direct_blocks;    /* renumbered pull only: local rows with a single edge whose source
                                 lies in the first `direct_blocks` blocks leave the blocked CSR
                                 (direct pieces, below); 0 = none, -1 = the blocks whose
                                 contributions fill at most 1/8 of the L2 */
} tc_part_params;

/*
 * Vertex order of a pull partition.  The paper cuts blocks as ranges of the graph's own
 * vertex IDs (Sec. 3.1).  TC_ORDER_OUTDEGREE first renumbers the vertices by out-degree,
 * highest first (ties by ID; among the vertices without out-edges, those without any edge
 * come last), and cuts the source ranges, local rows and merge ranges in that numbering:
 * the sources that feed most destinations then share blocks, so each destination has fewer
 * (block, row) pieces and the partial-sum traffic of the merge shrinks; the blocks past the
 * last vertex with out-edges would hold no edges and are dropped.  The merge ranges are cut
 * to hold about equal work (at most merge_range vertices each, merge_range >= 128) and cover
 * only the vertices with some edge; the rest all get the rank of an empty sum, set in closed
 * form.  Everything the caller sees stays
 * in the graph's own numbering: PageRank takes `init` and returns ranks by original ID.
 * tc_part_export reports the renumbered structure and tc_part_export_order the numbering.
 * Direct pieces: in a renumbered pull partition most (block, row) pieces of the first blocks -
 * the sources with the most out-edges - hold a single edge.  Such a piece's partial sum is
 * just its source's contribution, so it leaves the blocked CSR (and the gather) and the merge
 * adds that contribution itself, read from the contribution array (those blocks' values stay
 * in L2): 4 bytes of source ID and 2 of local target instead of a staged edge, a row start,
 * a partial sum written and read, and its 2-byte ID.  tc_part_export then reports the
 * blocked CSR without them (num_direct in tc_part_info counts them); with direct_blocks = 0 (the
 * default) it is the paper's blocking exactly.  Measured on R-MAT 24 the option is slower: the
 * gather gains 7-14% but the merge's random reads of the contribution array and its atomics on
 * a target's adjacent pieces cost more (see the design notes), so it stays off by default.
 * BFS and the PPR batch do not take renumbered partitions (TC_ERR_UNSUPPORTED), and push
 * partitions cannot be renumbered (TC_ERR_UNSUPPORTED).
 */
#define TC_ORDER_NATURAL    0
#define TC_ORDER_OUTDEGREE  1

/* tc_tocab_partition -- build the static 1D blocking described above (Sec. 3.1, Fig. 3/4), the
 * merge range table of Fig. 5 and, for pull partitions that fit, the staged format.  `out`
 * receives a library-owned handle (free with tc_part_free); the graph must outlive it.
 * Synchronises.  Errors as listed above, plus TC_ERR_UNSUPPORTED for more than 65,535 blocks or
 * smem_stage = 1 with a width that does not fit. */
int tc_tocab_partition(const tc_graph *g, int dir, int32_t num_blocks,
                       const tc_part_params *params /* NULL = defaults */, void *stream,
                       tc_part **out);
/* Release a partition; NULL is ignored (handle management, no counterpart in the paper). */
void tc_part_free(tc_part *p);

typedef struct tc_part_info {
    int32_t dir;
    int32_t num_blocks;       /* B */
    int32_t block_width;      /* W */
    int64_t num_rows;         /* R = sum over blocks of local rows */
    int64_t num_edges;        /* E */
    int32_t merge_range;      /* k */
    int32_t num_hubs;         /* rows handled one CTA per row */
    int32_t staged;           /* 1: the gather stages block contributions in shared memory */
    int64_t staged_edges;     /* edges of the staged stream incl. per-block padding (0 if not) */
    int32_t vertex_order;     /* TC_ORDER_NATURAL or TC_ORDER_OUTDEGREE */
    int32_t num_ranges;       /* merge ranges (CTAs of the merge) */
    int32_t num_tiles;        /* CTAs of the staged gather (0 if not staged) */
    int32_t num_sources;      /* vertices with out-edges (TC_ORDER_OUTDEGREE: they come first) */
    int32_t direct_blocks;    /* blocks whose single-edge pieces are direct (0: none) */
    int64_t num_direct;       /* direct pieces (not in num_rows / num_edges) */
} tc_part_info;
/* Shape of a partition: B and W of Sec. 3.1, R local rows (Fig. 4), k of Fig. 5.  Errors:
 * TC_ERR_INVALID_ARG for a NULL argument. */
int tc_part_get_info(const tc_part *p, tc_part_info *info);

/*
 * tc_part_export -- copy the blocked CSR of Sec. 3.1 (Fig. 3, local IDs of Fig. 4) out to
 * caller-owned buffers (mem = host or device), for inspection:
 *   blk_rows[B+1]  first local row of each block;   blk_edges[B+1] first edge of each block
 *   rowptr[R+1]    edge offset of every local row;  id_map[R] global ID of every local row
 *   colidx[E]      global column (source for pull, destination for push) of every edge.
 * Any output pointer may be NULL to skip it.  Synchronises.
 */
int tc_part_export(const tc_part *p, int64_t *blk_rows, int64_t *blk_edges, int32_t *rowptr,
                   int32_t *id_map, int32_t *colidx, int mem, void *stream);

/*
 * tc_part_export_order -- the vertex numbering of a partition (no counterpart in the paper;
 * see TC_ORDER_OUTDEGREE above): perm[n] = original ID of the vertex numbered n, V entries, to
 * a caller-owned buffer in `mem` space.  For a TC_ORDER_NATURAL partition perm[n] = n.  The IDs
 * that tc_part_export reports are the numbers n.  Synchronises.  Errors: TC_ERR_INVALID_ARG
 * (NULL partition or output, bad mem), TC_ERR_CUDA.
 */
int tc_part_export_order(const tc_part *p, int32_t *perm, int mem, void *stream);

/* Per-subgraph load balancing (Sec. 3.2, chosen per subgraph by the cost model):
 * warp_min_per_block (host int32[B], each >= 1, copied) replaces tc_pr_params.lb_warp_min for
 * the unstaged gathers of this partition; NULL clears it.  Errors: TC_ERR_INVALID_ARG (NULL
 * partition, an entry < 1), TC_ERR_OOM, TC_ERR_CUDA. */
int tc_part_set_lb(tc_part *p, const int32_t *warp_min_per_block);

/* Default block width W for a vertex count V and an L2 size: the rule used when num_blocks == 0,
 * W FP32 values in l2_fraction of the L2 (Sec. 4.3's 256 Ki vertices on a 2.75 MB L2, pinned by
 * Table 3).  Host-only and never fails: W is at least 32, and at most V when V > 0. */
int32_t tc_default_block_width(int32_t V, int64_t l2_bytes, float l2_fraction);

/* ---- PageRank ------------------------------------------------------------------------------ */
#define TC_MERGE_FIXED    0          /* one accumulator per CTA, exact fixed-point adds (two
                                        32-bit shared reductions per partial below 1,024
                                        blocks, three from 1,024): deterministic; the default,
                                        fastest measured on GB300                             */
#define TC_MERGE_ORDERED  1          /* per-warp FP32 accumulators added in a fixed order:
                                        deterministic; when 16 accumulators of merge_range
                                        floats do not fit in shared memory the call uses
                                        TC_MERGE_FIXED instead                                 */
/* (2 was an FP32-atomic merge; it could miss the 1e-5 accuracy bar on ranges with hundreds of
   pieces per vertex, measured slower, and is no longer accepted: TC_ERR_INVALID_ARG)         */
#define TC_PUSH_FLOAT     3          /* push only: FP32 atomicAdd into the sums (the paper's
                                        Alg. 2/5; order-dependent rounding).  Push otherwise
                                        (TC_MERGE_FIXED or _ORDERED) adds 64-bit fixed-point
                                        integers (red.add.u64): exact in any order, so the
                                        ranks repeat bit for bit                               */

typedef struct tc_pr_params {
    float   damping;          /* d, e.g. 0.85 */
    int32_t iters;            /* fixed number of Jacobi iterations (>= 0) */
    int32_t dangling;         /* TC_DANGLING_REDISTRIBUTE or TC_DANGLING_DROP */
    int32_t out_mem;          /* memory space of ranks_out (and of init) */
    const float *init;        /* initial ranks [V] or NULL for 1/V */
    int32_t profile;          /* nonzero: time each kernel with CUDA events (stats) */
    int32_t merge_mode;       /* TOCAB pull merge: TC_MERGE_FIXED (0) or TC_MERGE_ORDERED;
                                 push sums: fixed point (0, 1) or TC_PUSH_FLOAT */
    int32_t lb_warp_min;      /* unstaged gathers (Sec. 3.2): rows with fewer edges are summed
                                 by one lane, longer rows by a warp (hubs by a CTA); 0 = 32,
                                 1 = a warp for every row, large = lane-serial; a partition's
                                 per-block table (tc_part_set_lb) overrides it.  Push: 0 = an
                                 edge-parallel scatter (a thread per edge, the default; with a
                                 partition whose destination range fits shared memory, the
                                 staged scatter of tc_push.cu), > 0 = that thread/warp/CTA row
                                 mapping (TWC) with this threshold */
    int32_t l2_window;        /* nonzero: unstaged pull gathers (unblocked, or a partition without
                                 the staged format) run with an L2 access-policy window over the
                                 contributions they read, so that the cache keeps the block's
                                 vertex values (Sec. 3.1) while the edges stream past.  The
                                 context's persisting L2 set-aside is raised for the call and
                                 restored before it returns, and the call synchronises the stream.
                                 A device without a set-aside runs the call without a window.
                                 Results are bitwise those of l2_window = 0 */
} tc_pr_params;

typedef struct tc_pr_stats {
    int32_t iters;            /* iterations run */
    int32_t launches;         /* kernels launched by the call */
    float   ms_total;         /* device time of the whole call (profile only) */
    float   ms_gather;        /* device time of gather/scatter kernels (profile only) */
    float   ms_merge;         /* device time of merge/update kernels (profile only) */
    double  dangling_mass;    /* dangling mass D of the final ranks */
} tc_pr_stats;

/*
 * tc_pagerank_pull -- PageRank in the pull direction.  Alg. 1 per iteration:
 *   contributions[u] = rank[u] / out_degree[u];  sums[v] = sum_{u -> v} contributions[u];
 *   rank[v] = (1-d)/|V| + d * (sums[v] + D/|V|)   (D = dangling mass, REDISTRIBUTE mode)
 * part == NULL runs the unblocked kernel (one gather over G^T with the update fused).
 * part != NULL (TC_PULL) runs TOCAB: Alg. 4 per block into dense partial sums over local
 * IDs, then the merge of Fig. 5 (CTA per vertex range) fused with the update.
 * All blocks read the previous iteration's contributions (Jacobi).  FP32 arithmetic.
 *   ranks_out : [V] floats in params->out_mem space.
 * Errors: TC_ERR_INVALID_ARG (null graph/params/output, damping outside [0,1], iters < 0,
 * partition of another graph or direction), TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_pagerank_pull(const tc_graph *g, const tc_part *part, const tc_pr_params *params,
                     float *ranks_out, tc_pr_stats *stats, void *stream);

/*
 * tc_pagerank_push -- PageRank in the push direction.  Alg. 2: every source scatters its
 * contribution into sums[dst] with atomic adds; part == NULL scatters over all of G,
 * part != NULL (TC_PUSH) runs Alg. 5 block by block, so that the atomics of one block
 * land in its destination range; then the same update as Alg. 1.  Summation order of
 * the atomics is not deterministic.  Same arguments and errors as tc_pagerank_pull.
 */
int tc_pagerank_push(const tc_graph *g, const tc_part *part, const tc_pr_params *params,
                     float *ranks_out, tc_pr_stats *stats, void *stream);

/* ---- BFS --------------------------------------------------------------------------------------- */
typedef struct tc_bfs_params {
    float   tocab_threshold;  /* use the blocked kernel in levels whose frontier holds more
                                 than this fraction of V (Sec. 3.3); < 0 = never, 0 = always */
    int32_t out_mem;          /* memory space of levels_out */
    int32_t profile;          /* nonzero: per-kernel device timing into stats */
    float   push_threshold;   /* 0 = every level pulls (topology-driven, the default); > 0 =
                                 direction optimisation, the push phases of the push-pull-push
                                 schedule of Sec. 3.3: start top-down (data-driven queue),
                                 switch to pull when the frontier's out-edges exceed 1/14 of
                                 the unvisited vertices' out-edges, and back to push when the
                                 frontier holds fewer than push_threshold * V vertices */
    int32_t resident_edges;   /* push levels only: consecutive levels whose frontier has at most
                                 this many vertices and out-edges run inside ONE launch of a
                                 thread-block cluster (16 CTAs, else 8), the levels ended by the
                                 cluster barrier instead of a host round trip (device memory:
                                 24 x cluster size x resident_edges bytes, kept with the graph);
                                 the frontier bitmap is rebuilt from the queue before the next
                                 pull level.
                                 No counterpart in the paper (its levels are host-driven): it
                                 serves the long-diameter graphs' thousands of small levels.
                                 0 = off, < 0 = TC_BFS_RESIDENT_DEFAULT, at most
                                 TC_BFS_RESIDENT_MAX (else TC_ERR_INVALID_ARG); levels are
                                 identical either way */
} tc_bfs_params;

#define TC_BFS_RESIDENT_DEFAULT 65536
#define TC_BFS_RESIDENT_MAX (1 << 20)

#define TC_BFS_TRACE 64
typedef struct tc_bfs_stats {
    int32_t levels;           /* number of BFS levels expanded (depth + 1 of the deepest) */
    int32_t tocab_levels;     /* levels run with the blocked kernel */
    int64_t reached;          /* vertices with level >= 0 */
    int64_t edges_reached;    /* sum of out-degrees of reached vertices */
    float   ms_total;         /* device time (profile only) */
    int32_t push_levels;      /* levels run top-down */
    /* first TC_BFS_TRACE levels: kind (0 pull, 1 pull TOCAB, 2 push, 3 push inside a resident
       launch), frontier size at the start of the level, device time (profile only; a resident
       launch's time is shared evenly by its levels) */
    int32_t level_kind[TC_BFS_TRACE];
    int64_t level_frontier[TC_BFS_TRACE];
    float   level_ms[TC_BFS_TRACE];
    int32_t resident_levels;  /* push levels run inside resident launches (counted in push_levels) */
} tc_bfs_stats;

/*
 * tc_bfs_pull -- topology-driven, level-synchronous BFS in the pull direction with
 * bitmap status arrays (front, next, visited; Sec. 3.3, Fig. 1e/f): in level L every
 * unvisited vertex v scans its in-edges and joins level L+1 if an in-neighbour is in
 * the frontier.  With part != NULL (TC_PULL) levels whose frontier exceeds the threshold
 * run per block into local next bitmaps over local IDs, OR-reduced in the merge kernel
 * (Sec. 3.3).  With push_threshold > 0, small-frontier levels run top-down from a queue
 * instead (direction optimisation); levels are identical either way.
 * levels_out[v] = hop distance from `source`, -1 when unreachable.
 * Errors: TC_ERR_INVALID_ARG (source outside [0, V)), TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_bfs_pull(const tc_graph *g, const tc_part *part, int32_t source,
                const tc_bfs_params *params, int32_t *levels_out, tc_bfs_stats *stats,
                void *stream);

/* ---- batched personalised PageRank -------------------------------------------------------- */
/*
 * tc_ppr_batch -- personalised PageRank for n sources in one batch (one column per source).
 * Column j runs Alg. 1 with the teleport (1-d) and the dangling mass of the column both sent
 * to its source s_j, starting from e_{s_j}:
 *   R'[v,j] = d * sum_{u->v} R[u,j] / out_degree[u] + [v == s_j] ((1-d) + d * D_j),
 *   D_j = sum of R[u,j] over dangling u.
 * The batch lives as an FP32 [V x n] row-major matrix.
 *   part == NULL : all iterations run as ONE persistent cooperative launch (one grid barrier
 *                  per iteration), captured in a CUDA graph that later calls with the same output
 *                  buffer, n, iters, damping and tuning replay.  The batch works in the graph's
 *                  vertex numbering by out-degree (built on first use and kept with the graph):
 *                  the rows of the sources with the most out-edges are one contiguous block.
 *                  The columns run in tiles of 32, 64 or 128 (all iterations of one tile, then
 *                  the next), or as whole rows; a lane group reads the tile's segment of a
 *                  source row per in-edge, so a smaller tile lets the L2 hold more source rows
 *                  (the source block sized to the cache of Sec. 3.1, without partial sums).
 *                  Warps draw work from a queue: pieces of the rows with more than 2048
 *                  in-edges, then runs of rows each walked as one in-edge stream.  Loads and
 *                  stores of the first `hot` rows carry an L2 evict-last priority, every other
 *                  row and the in-edge lists evict-first.  Tile width and `hot` come from
 *                  tc_ppr_autotune when it has run, else 32 columns and half the rows the L2
 *                  holds.
 *   part != NULL : TOCAB per column tile (Sec. 3.1): columns in tiles of 32; for each tile,
 *                  Alg. 4 over the partition's source blocks (size them so that W x 128 bytes
 *                  of a block's row segments fit in L2, e.g. l2_fraction = 1/88) into 32-wide
 *                  partial rows, then the Fig. 5 merge (blocks added in order; deterministic)
 *                  with the update.  The partition's merge_range k must be <= 1600 (256 advised).
 *   sources : host int32[n], each in [0, V) (repeats allowed);  1 <= n <= 1024.
 *   params  : damping, iters, out_mem (R_out space), profile (stats->ms_total); init ignored.
 *   R_out   : float[V * n], R_out[v*n + j].
 * Device scratch: two [V x round_up(n,128)] FP32 matrices (part == NULL: kept with the graph
 * for later calls with the same padded width; otherwise allocated and freed per call).
 * Synchronises the stream before returning.
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED (n out of range, or a renumbered partition),
 * TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT (a grid barrier gave up after about a second).
 */
int tc_ppr_batch(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t n,
                 const tc_pr_params *params, float *R_out, tc_pr_stats *stats, void *stream);

/*
 * tc_ppr_autotune -- times the persistent batch (part == NULL above) for this graph and batch
 * width over its tile width (whole rows, 128, 64 or 32 columns) and the size of its evict-last
 * block (0, 1/4, 1/2 or all of the rows of that width the L2 holds), on `sources` with
 * params->iters capped at 3, and keeps the fastest with the graph for later tc_ppr_batch calls
 * (no counterpart in the paper, which sizes its blocks from the cache size alone).
 *   best_hot  : the chosen evict-last rows (may be NULL).
 *   best_tile : the chosen tile width in columns, 0 for whole rows (may be NULL).
 *   times     : float[16] or NULL: ms of each variant, tile-major (whole, 128, 64, 32) x
 *               evict-last fraction (0, 1/4, 1/2, 1).
 * Synchronises.  Errors: as tc_ppr_batch.
 */
int tc_ppr_autotune(tc_graph *g, const int32_t *sources, int32_t n, const tc_pr_params *params,
                    int32_t *best_hot, int32_t *best_tile, float *times, void *stream);

/*
 * tc_ppr_set_tuning -- sets the persistent batch's schedule for this graph by hand, as
 * tc_ppr_autotune would (no counterpart in the paper): hot = evict-last rows (clamped to what the L2 holds; -1: the default),
 * tile = 0 (whole rows), 32, 64 or 128 columns (-1: the default).  Results do not depend on
 * hot; the tile width changes how each row's in-edges are grouped for summation (rounding only).
 * Errors: TC_ERR_INVALID_ARG.
 */
int tc_ppr_set_tuning(tc_graph *g, int32_t hot, int32_t tile);

/* ---- betweenness centrality ----------------------------------------------------------------- */
/*
 * tc_bc_forward -- the shortest-path calculation of Alg. 3 from one source over the out-edges
 * of G: depth_out[v] = hop distance from `source` (-1 when unreachable; the paper's delta) and
 * sigma_out[v] = number of shortest paths from `source` to v (the paper's sigma, FP64, exact
 * below 2^53; 0 when unreachable).  Each level runs in the cheaper direction (Sec. 3.3's
 * push-pull-push): push over the frontier's out-edges, edge-balanced (compare-and-swap on depth,
 * FP64 atomics on sigma - exact, as every partial sum is an integer below 2^53) while those
 * edges are fewer than 1/14 of the out-edges of the vertices not yet reached (Beamer's rule),
 * else pull over the in-rows of the unreached vertices (a thread per short row, a warp per row
 * of 32 or more in-edges).  Results do not depend on the direction chosen.
 *   out_mem : memory space of depth_out (int32[V]) and sigma_out (double[V]).
 * Synchronises the stream.  Errors: TC_ERR_INVALID_ARG (source outside [0, V), bad out_mem),
 * TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_bc_forward(const tc_graph *g, int32_t source, int out_mem, int32_t *depth_out, double *sigma_out,
                  void *stream);

/*
 * tc_bc -- betweenness-centrality scores from a set of sources (Sec. 3.3's BC benchmark): for
 * each source, Alg. 3's forward sweep, then the dependency back-propagation over the levels in
 * reverse,
 *   dep[v] = sum over out-neighbours w with depth[w] = depth[v] + 1 of sigma[v]/sigma[w] (1 + dep[w]),
 * pulled over the out-edges of G; scores_out[v] = the sum of dep[v] over the sources other than
 * v itself.  Scores are not normalised and count ordered targets (an undirected graph given
 * with both edge directions counts every pair twice).  FP64 throughout, computed as
 * dep[v] = sigma[v] * sum over w of (1 + dep[w]) / sigma[w] (one division per vertex); every
 * product, quotient and sum is rounded separately.  A vertex's out-row is summed by 8 lanes (up
 * to 64 edges), a warp (up to the graph's hub degree, 2048) or a CTA (above it), each lane in
 * strided order and a fixed shuffle or block tree adding the lanes, so the result is
 * deterministic.
 *   sources : host int32[num_sources], each in [0, V) (repeats allowed; 0 sources gives zeros).
 *   out_mem : memory space of scores_out (double[V]).
 * Scratch: 3 int32[V] + int64[V] + 3 double[V] (+ double[V] for host output), per call.
 * Synchronises the stream.  Errors: TC_ERR_INVALID_ARG, TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_bc(const tc_graph *g, const int32_t *sources, int32_t num_sources, int out_mem, double *scores_out,
          void *stream);

/*
 * tc_bc_tocab -- tc_bc with TOCAB in the pull levels of the forward sweep (Sec. 3.3: the
 * push-pull-push BC with blocked pull levels, where "next" carries the sigma sums of the block's
 * local rows): each local row of the partition sums sigma over its sources of depth L, then the
 * merge of Fig. 5 adds a destination's pieces in block order (integers: exact), so depths, sigma
 * and the scores equal tc_bc's bit for bit.
 *   part : a TC_PULL partition of g in the graph's own numbering (TC_ERR_UNSUPPORTED for a
 *          renumbered one), merge_range at most 25,600.
 * Scratch: as tc_bc, plus double[R].  Errors: as tc_bc.
 */
int tc_bc_tocab(const tc_graph *g, const tc_part *part, const int32_t *sources, int32_t num_sources, int out_mem,
                double *scores_out, void *stream);

/* ---- sparse matrix-vector product ---------------------------------------------------------- */
/*
 * tc_spmv -- y = A x (the SpMV benchmark of Sec. 4).  A is the CSR loaded with
 * tc_graph_load_csr, read as rows = outputs: y[i] = sum over the stored entries k of row i of
 * vals[k] * x[colidx[k]], with vals in the loaded entry order.  FP32 values, vectors and
 * accumulation; a group of 4 to 32 lanes per row (from the mean row length) and a CTA per row
 * of more than the hub degree (Sec. 3.2's binning), each with a fixed reduction order
 * (deterministic).  The graph's transpose is not used.
 *   vals : float[E], x : float[V], y : float[V] (y[i] for every row i < V), all device pointers.
 *   mem  : TC_MEM_DEVICE (TC_MEM_HOST is refused with TC_ERR_UNSUPPORTED).
 * Asynchronous on `stream`.  Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED, TC_ERR_CUDA.
 */
int tc_spmv(const tc_graph *g, const float *vals, const float *x, float *y, int mem, void *stream);

/*
 * tc_part_set_values -- give a partition of the matrix's graph the values of the stored entries,
 * `vals` in the loaded CSR order (float[E], device).  A TC_PUSH partition's blocks are ranges of
 * W columns of A and its local rows the (column block, row) pieces of Fig. 4 (GC-pull SpMV); a
 * TC_PULL partition's blocks are ranges of W rows of A and its local rows the (row block,
 * column) pieces (GC-push SpMV).  The partition keeps the values in its own entry order (the
 * first call also records that order: the partition's stable sorts again, carrying entry
 * positions).  For the SpMV of Sec. 4.  Synchronises.
 * Errors: TC_ERR_INVALID_ARG (NULL), TC_ERR_UNSUPPORTED (host values, a renumbered partition),
 * TC_ERR_OOM, TC_ERR_CUDA.
 */
int tc_part_set_values(tc_part *p, const float *vals, int mem, void *stream);

/*
 * tc_spmv_tocab -- y = A x with TOCAB (the SpMV of Sec. 4, a value stream of 4 B per entry).
 *   TC_PUSH partition: GC-pull.  For every local row (column block b, row i), partial = sum of
 *       vals * x[col] over the piece's entries (x's block b is the working set, Sec. 3.1), then
 *       the merge of Fig. 5 adds row i's pieces in block order.  FP32 in a fixed order
 *       (deterministic).  The merge_range k must be at most 51,200.
 *   TC_PULL partition (graph's own numbering): GC-push.  y = 0, then for every local row (row
 *       block b, column j) each entry (i, j) adds vals * x[j] into y[i] with an FP32 atomic add
 *       (y's block b is the working set).  The order of the additions depends on timing, so the
 *       last bits of y may differ between calls; each y[i] is within the FP32 summation bound.
 *   In both, a lane takes a piece below 32 entries, a warp a longer one (Sec. 3.2).
 *   p : a partition of the graph holding A, with values set by tc_part_set_values.
 *   x : float[V], y : float[V], device.
 * Asynchronous on `stream`.  Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED, TC_ERR_CUDA.
 */
int tc_spmv_tocab(const tc_part *p, const float *x, float *y, int mem, void *stream);

/* ---- many small graphs in one batch ---------------------------------------------------------- */
typedef struct tc_multigraph tc_multigraph;   /* opaque: a batch of independent graphs */

/*
 * tc_multigraph_load -- load a batch of independent graphs as one disjoint union.  Graph g
 * owns the vertices [vtx_off[g], vtx_off[g+1]); rowptr/colidx is the out-edge CSR of the union
 * in those global IDs (layout and rules as tc_graph_load_csr).  Every edge must join two
 * vertices of the same graph (TC_ERR_INVALID_GRAPH otherwise).
 *   vtx_off : host int32[num_graphs + 1], vtx_off[0] = 0, non-decreasing, vtx_off[n] = V.
 * Batching of independent graphs has no counterpart in the paper; each graph runs Alg. 1.
 * Errors: those of tc_graph_load_csr, TC_ERR_INVALID_ARG for a bad vtx_off.
 */
int tc_multigraph_load(int32_t num_graphs, const int32_t *vtx_off, int32_t V, int64_t E,
                       const int32_t *rowptr, const int32_t *colidx, int mem, void *stream,
                       tc_multigraph **out);
/* Release a batch; NULL is ignored (handle management, no counterpart in the paper).  Waits for
 * the device before freeing. */
void tc_multigraph_free(tc_multigraph *m);

#define TC_MULTI_RESIDENT 1024    /* lanes_per_vertex value: each graph stays in one CTA for all
                                     iterations, its contributions in shared memory (needs every
                                     graph's non-dangling vertex count to fit; TC_ERR_UNSUPPORTED
                                     otherwise)                                                  */
typedef struct tc_multi_params {
    int32_t lanes_per_vertex; /* 0 = the autotuned choice (hybrid until tuned), -1 = a lane per
                                 vertex with rows of 32+ edges taken by the warp, 1/4/8/32, or
                                 TC_MULTI_RESIDENT */
    int32_t ctas_per_sm;      /* 0 = as many as fit (then the launch is graph-captured) */
    int32_t use_graph;        /* 1 = launch through the cached captured CUDA graph */
} tc_multi_params;

/*
 * tc_pagerank_multi -- Alg. 1 on every graph of the batch at once; graph g uses its own
 * teleport (1-d)/V_g and its own dangling mass D_g (redistributed over its own vertices).
 * All iterations run in one persistent cooperative kernel with a grid barrier between them
 * (a bounded spin: TC_ERR_TIMEOUT if it ever gives up), or, for TC_MULTI_RESIDENT, in one
 * kernel whose CTAs each run a whole graph; with use_graph the launch is captured once into a
 * CUDA graph (cached in the handle per parameter set) and replayed.
 *   ranks_out : float[V] (params->out_mem), in the union's vertex order.  params->init must
 *               be NULL (TC_ERR_UNSUPPORTED otherwise).
 * Errors: TC_ERR_INVALID_ARG, TC_ERR_UNSUPPORTED, TC_ERR_TIMEOUT, TC_ERR_CUDA.
 */
int tc_pagerank_multi(const tc_multigraph *m, const tc_pr_params *params, const tc_multi_params *mp,
                      float *ranks_out, tc_pr_stats *stats, void *stream);

/*
 * tc_multi_autotune -- the project's autotuner for the batch (no counterpart in the paper; the
 * variants are the thread/warp mappings of Sec. 3.2 plus the resident form): times every lanes-per-vertex
 * variant (-1, 1, 4, 8, 32, and TC_MULTI_RESIDENT when the graphs fit; one warm-up and one
 * timed run each, CUDA events) with `params`, stores the fastest in the handle (used when
 * lanes_per_vertex = 0) and returns it.
 *   times_ms : optional float[6], time of each variant in the order -1, 1, 4, 8, 32,
 *              TC_MULTI_RESIDENT (a negative time: the variant does not apply to this batch).
 */
int tc_multi_autotune(tc_multigraph *m, const tc_pr_params *params, int32_t *best_lanes,
                      float *times_ms, void *stream);

/* ---- learned cost model ------------------------------------------------------------------------ */
/*
 * Features (16 floats) of a graph or of a TOCAB subgraph, computed on the device from its rows
 * (destinations for pull): log2 rows, log2 edges, mean degree, degree coefficient of
 * variation, log2(1 + max/mean degree), fractions of rows with degree 0, 1-7, 8-15, 16-31 and
 * 32+ (the bins of the paper's Table 1), out-degree coefficient of variation, dangling
 * fraction, log2(1 + vertex-value bytes / L2), log2(1 + column-index bytes / L2), ID locality
 * (mean |first source - row| / V), log2(1 + max/mean out-degree).  Synchronises.
 */
int tc_graph_features(const tc_graph *g, float *features /* host [16] */);
/* Features of every block of a partition (the subgraphs of Sec. 3.1): host float[B][16] (the
 * out-degree features and the vertex-value bytes are the graph's and the block width's).
 * Synchronises.  Errors: TC_ERR_INVALID_ARG (NULL argument), TC_ERR_OOM, TC_ERR_CUDA. */
int tc_part_features(const tc_part *p, float *features);

/*
 * The cost model's network (no counterpart in the paper: it only picks parameters of the
 * method and never changes its results):  z = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3,
 * with the outputs split into `n_heads` softmax heads; loss = mean over samples of the summed
 * cross-entropy.  FP32, forward/backward/Adam in the library's own kernels; every reduction
 * over samples runs in a fixed order (deterministic).  Parameters are one flat float vector:
 * W1[n_in][n_hidden], b1, W2[n_hidden][n_hidden], b2, W3[n_hidden][n_out], b3 (row-major).
 */
typedef struct tc_mlp tc_mlp;
/* Create the network above (no counterpart in the paper) with zero parameters; `out` receives
 * a library-owned handle.  Errors: TC_ERR_INVALID_ARG (a size < 1, more than 8 heads, NULL head
 * sizes or out), TC_ERR_OOM, TC_ERR_CUDA. */
int tc_mlp_create(int32_t n_in, int32_t n_hidden, int32_t n_heads, const int32_t *head_sizes,
                  tc_mlp **out);
/* Release a network; NULL is ignored (no counterpart in the paper). */
void tc_mlp_free(tc_mlp *m);
/* Number of parameters of the flat vector (no counterpart in the paper); -1 for NULL. */
int64_t tc_mlp_num_params(const tc_mlp *m);
/* Set the parameters (host float[num_params]); resets the Adam moments (cost model, no
 * counterpart in the paper).  Errors: TC_ERR_INVALID_ARG, TC_ERR_CUDA. */
int tc_mlp_set_params(tc_mlp *m, const float *params);
/* Copy parameters and/or the last computed gradients to host, either may be NULL (cost model,
 * no counterpart in the paper).  Errors: TC_ERR_INVALID_ARG, TC_ERR_CUDA. */
int tc_mlp_get_params(const tc_mlp *m, float *params, float *grads);
/* Z[N][n_out] = network outputs (logits) for X[N][n_in]; X and Z in `mem` space (cost model, no
 * counterpart in the paper).  Errors: TC_ERR_INVALID_ARG, TC_ERR_OOM, TC_ERR_CUDA. */
int tc_mlp_forward(tc_mlp *m, const float *X, int32_t N, float *Z, int mem, void *stream);
/* Loss (host *loss) and gradients (kept in the handle) for X[N][n_in], labels Y[N][n_heads]
 * (cost model, no counterpart in the paper).  Every label must lie in [0, size of its head):
 * the labels are checked on the device before any kernel uses them, and a label outside its
 * head fails the call with TC_ERR_INVALID_ARG (nothing is updated).  Errors:
 * TC_ERR_INVALID_ARG (NULL argument, N < 1, label out of range), TC_ERR_OOM, TC_ERR_CUDA. */
int tc_mlp_loss_grad(tc_mlp *m, const float *X, const int32_t *Y, int32_t N, int mem,
                     double *loss, void *stream);
/* One Adam step (Kingma & Ba) with the gradients of the last tc_mlp_loss_grad (cost model, no
 * counterpart in the paper).  Errors: TC_ERR_INVALID_ARG, TC_ERR_CUDA. */
int tc_mlp_adam_step(tc_mlp *m, float lr, float beta1, float beta2, float eps, void *stream);
/* `epochs` passes of minibatch Adam (lr, beta 0.9/0.999, eps 1e-8) over the samples in the
 * given order; *final_loss = loss over all samples afterwards (cost model, no counterpart in the
 * paper).  Labels as for tc_mlp_loss_grad.  Errors: TC_ERR_INVALID_ARG, TC_ERR_OOM, TC_ERR_CUDA. */
int tc_mlp_train(tc_mlp *m, const float *X, const int32_t *Y, int32_t N, int32_t epochs,
                 int32_t batch, float lr, int mem, double *final_loss, void *stream);

/* ---- PageRank without allocation ------------------------------------------------------------ */
/* Largest vertex count and size in bytes of the static device scratch used below. */
#define TC_NOALLOC_MAX_V          (1 << 20)
#define TC_NOALLOC_SCRATCH_BYTES  (256 + 4096 * 8 + 3 * 4 * TC_NOALLOC_MAX_V)

/*
 * tc_pagerank_pull_noalloc -- the unblocked pull PageRank of tc_pagerank_pull for callers
 * that cannot allocate device memory (the paper has no counterpart: this entry point is a
 * deployment aid).  Typical callers run inside a host framework whose allocator owns the
 * device memory pool, or fix their memory budget at start-up and may not call cudaMalloc
 * or cudaFree afterwards.  This call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.  Its scratch (contributions, out-degree reciprocals,
 * dangling-mass partials) is a static device array of TC_NOALLOC_SCRATCH_BYTES (about
 * 12.6 MB) that every GPU which loads the library holds until the process exits.
 * Under CUDA's default lazy module loading, that array's device memory is reserved when
 * the library's module is first used on a device -- by the first call of this entry point
 * there -- so the first call can still fail with TC_ERR_CUDA when the device has no room
 * left.  A caller whose memory budget or pool is fixed later should make one call (any
 * valid V, iters = 0 will do) on every device at start-up, before the pool is taken, or
 * load modules eagerly (environment CUDA_MODULE_LOADING=EAGER).  Later calls reserve nothing.
 *   V          : 1 <= V <= TC_NOALLOC_MAX_V, else TC_ERR_UNSUPPORTED (nothing is launched).
 *   in_rowptr  : device int32[V+1], in-edge CSR of G^T (row v lists the sources of v's
 *   in_colidx    in-edges; device int32[E]).  Not validated: pass a well-formed CSR.
 *   out_degree : device int32[V], out-degree of every vertex in G.
 *   damping, iters, dangling : as tc_pr_params (TC_DANGLING_REDISTRIBUTE or _DROP).
 *   ranks_out  : device float[V], receives the ranks after `iters` iterations.
 *   stream     : cudaStream_t; the call only enqueues work on it and does not synchronise.
 * The first call on a device looks up the scratch's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  All calls
 * share the one scratch array, which keeps the previous call's contents (the call re-arms
 * what must start at zero): calls whose work overlaps on the GPU -- on different streams,
 * or from different threads -- race and give wrong results; serialise them.
 * Errors: TC_ERR_UNSUPPORTED (V out of range), TC_ERR_INVALID_ARG (null pointer, damping
 * outside [0,1], iters < 0, bad dangling mode), TC_ERR_CUDA (launch or lookup failure).
 */
int tc_pagerank_pull_noalloc(int32_t V, const int32_t *in_rowptr, const int32_t *in_colidx,
                             const int32_t *out_degree, float damping, int32_t iters,
                             int32_t dangling, float *ranks_out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TOCAB_H */
