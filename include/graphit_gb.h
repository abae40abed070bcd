/*
 * graphit_gb.h -- C ABI of the GB300 edgeset-apply library.
 *
 * The operations follow the operator API of GraphIt (Zhang et al., OOPSLA 2018):
 * the vertexset/edgeset operators of Table 2 (size, from, to, srcFilter,
 * dstFilter, apply, applyModified with optional deduplication) and the
 * scheduling choices of Table 3 (configApplyDirection, configApplyParallelization,
 * configApplyDenseVertexSet, configApplyNumSSG), executed by hand-written CUDA
 * kernels for sm_103a.
 *
 * Conventions for every call:
 *   - The return value is a status: GI_OK (0) or a negative GI_ERR_* code.  No
 *     exception or abort crosses the ABI.  gi_last_error() returns a message for
 *     the calling thread's most recent failure.
 *   - "dev" pointers are CUDA device pointers owned by the caller; the library
 *     never frees them and reads/writes them only inside the call's stream order.
 *   - Handles (gi_graph, gi_vset) are owned by the library and released with the
 *     matching *_free call.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  Work is enqueued on it; calls documented as "syncs" wait for it.
 *   - Vertex ids and arc offsets are int32 (graphs with fewer than 2^31 arcs).
 *   - Threads: different graphs may be loaded and traversed from different
 *     host threads on different streams at the same time.  One graph runs one
 *     traversal at a time (its scratch lists, tiles and hot-source set are
 *     per graph); gi_graph_free and gi_vset_free synchronise the device.
 */
#ifndef GRAPHIT_GB_H
#define GRAPHIT_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status -- */
#define GI_OK 0
#define GI_ERR_INVALID_ARG (-1) /* NULL handle, bad size, unknown enum value        */
#define GI_ERR_BAD_GRAPH (-2)   /* CSR/CSC failed validation (GI_VALIDATE)           */
#define GI_ERR_OOM (-3)         /* device or pinned-host allocation failed           */
#define GI_ERR_CUDA (-4)        /* a CUDA runtime call or kernel launch failed       */
#define GI_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up                */
#define GI_ERR_UNSUPPORTED (-6) /* combination not implemented (e.g. m >= 2^31)      */

/* Message of the calling thread's last failure ("" if none).  Never NULL. */
const char *gi_last_error(void);
/* Library version as major*10000 + minor*100 + patch (never fails). */
int gi_version(void);

/* ----------------------------------------------------------------- graph -- */
typedef struct gi_graph gi_graph;

#define GI_HOST_PTRS 0x1u /* input arrays are host memory (copied host-to-device)            */
#define GI_DEV_PTRS 0x2u  /* input arrays are device memory (copied device-to-device)        */
#define GI_SYMMETRIC 0x4u /* every arc (u,v) has its reverse: the in-edge view aliases CSR   */
#define GI_VALIDATE 0x8u  /* check offsets/indices on the device; GI_ERR_BAD_GRAPH if bad    */
#define GI_HOT_SOURCES 0x10u /* also build the hot-source set of the dense pull during the load */

/*
 * Load a graph's out-edges in CSR form (the edgeset of Sec. 3; getOutNghs of the
 * generated code in Sec. 6).  offsets[n+1] (offsets[0] = 0, non-decreasing,
 * offsets[n] = m), indices[m] in [0,n), each row sorted ascending; weights[m] may
 * be NULL.  The arrays are copied: the caller may free them after the call
 * returns (the stream is synchronised before return).  Also builds out-degrees,
 * 1/out-degree and the pull tiles.  For GI_SYMMETRIC graphs the in-edge (CSC)
 * view is the CSR itself; otherwise call gi_load_csc before any pull traversal.
 * The indices (and weights) are copied on an internal stream in pieces, so
 * that the degree and tile work runs under the copy.  GI_HOT_SOURCES also
 * builds the hot-source set of the on-chip pull (gi_schedule.hot_cache,
 * otherwise built on first use) while the in-edges arrive, each piece
 * remapped as soon as it has landed; it takes effect on the call that loads
 * the in-edges (this one for GI_SYMMETRIC graphs, gi_load_csc otherwise).
 * Errors: GI_ERR_INVALID_ARG (n < 0, m < 0, NULL pointers with m > 0, both or
 * neither of HOST/DEV flags), GI_ERR_UNSUPPORTED (n or m >= 2^31),
 * GI_ERR_BAD_GRAPH (GI_VALIDATE and a check failed), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_load_csr(const int32_t *offsets, const int32_t *indices, const int32_t *weights, int64_t n, int64_t m,
                uint32_t flags, void *stream, gi_graph **out);

/*
 * Attach the in-edges (CSC: getInNghs of Sec. 6) of a non-symmetric graph:
 * in_offsets[n+1], in_indices[m] (sources, sorted ascending per row),
 * in_weights[m] or NULL.  Same copy, flag and error rules as gi_load_csr.
 */
int gi_load_csc(gi_graph *g, const int32_t *in_offsets, const int32_t *in_indices, const int32_t *in_weights,
                uint32_t flags, void *stream);

/* Releases g and everything built on it (tiles, segments, caches); NULL is a no-op. */
int gi_graph_free(gi_graph *g);

/* n, m and the maximum out-degree (host outputs).  Any output pointer may be
 * NULL.  Errors: GI_ERR_INVALID_ARG (g NULL). */
int gi_graph_info(const gi_graph *g, int64_t *n, int64_t *m, int32_t *max_deg);

/*
 * The hot-source set of the on-chip pull (gi_schedule.hot_cache), built on
 * first use from the in-edges (this call builds it, syncing `stream`): *k
 * sources, those of out-degree >= *min_deg, where min_deg is the smallest
 * threshold with at most 24,576 sources (k = 0, min_deg = 0 for a graph
 * without arcs); their slots follow descending degree.  Errors:
 * GI_ERR_UNSUPPORTED without in-edges, GI_ERR_OOM.
 */
int gi_graph_hot_info(gi_graph *g, int32_t *k, int32_t *min_deg, void *stream);

/* Device pointers of the library's copy: out-offsets, out-indices, out-weights (NULL if none);
 * owned by g, valid until gi_graph_free.  Errors: GI_ERR_INVALID_ARG (g NULL). */
int gi_graph_device_csr(const gi_graph *g, const int32_t **offsets, const int32_t **indices,
                        const int32_t **weights);

/*
 * Build the segmented subgraphs (SSGs) used by segmented pull (cache
 * partitioning, Sec. 2 and the SSG code generation of Sec. 6): the in-edges are
 * split into num_segments groups by source range, each sorted by destination.
 * strategy GI_SEG_FVC (fixed vertex count): segment s keeps the sources
 * [s*ceil(n/S), (s+1)*ceil(n/S)); GI_SEG_EVC (edge-aware vertex count): the
 * ranges are cut where the prefix sum of the sources' out-degrees crosses
 * s*m/S, so each segment holds about m/S arcs (one source never splits).
 * num_segments = 1 frees them.  Kept until the next call or gi_graph_free.
 * Errors: GI_ERR_INVALID_ARG, GI_ERR_UNSUPPORTED (no in-edges), GI_ERR_OOM
 * (nothing is kept then).
 */
#define GI_SEG_FVC 0
#define GI_SEG_EVC 1
int gi_graph_build_segments(gi_graph *g, int32_t num_segments, int32_t strategy, void *stream);

/*
 * The current segments (host memory outputs): *num (1 without segments),
 * *strategy, bounds[0..num] (segment s holds sources [bounds[s], bounds[s+1]))
 * and arcs[0..num-1]; any output may be NULL, and at most cap segments are
 * written.  Does not touch the device.  Errors: GI_ERR_INVALID_ARG (g NULL).
 */
int gi_graph_segment_info(const gi_graph *g, int32_t *num, int32_t *strategy, int32_t *bounds, int64_t *arcs,
                          int32_t cap);

/* ------------------------------------------------------------- vertexset -- */
typedef struct gi_vset gi_vset;

#define GI_VSET_EMPTY 0  /* no vertex                          */
#define GI_VSET_ALL 1    /* every vertex (edges.getVertices())  */
#define GI_VSET_SINGLE 2 /* the single vertex `v`               */

/* Representations (Sec. 2 "Direction Optimization and Frontier Data Structure"). */
#define GI_REP_SPARSE 0x1u /* array of vertex ids + count (SparsePush frontier)      */
#define GI_REP_BOOL 0x2u   /* one byte per vertex (boolean map)                      */
#define GI_REP_BITMAP 0x4u /* one bit per vertex, uint32 words (bitvector)           */

/* Create a vertexset over g's vertices (init GI_VSET_*, v for SINGLE); it stays
 * valid until gi_vset_free and must be freed before g.  Errors:
 * GI_ERR_INVALID_ARG (NULL g/out, unknown init, v out of range), GI_ERR_OOM. */
int gi_vset_create(gi_graph *g, int32_t init, int32_t v, void *stream, gi_vset **out);
/* Releases s (NULL is a no-op). */
int gi_vset_free(gi_vset *s);

/* size() of Table 2 into *out (host).  Syncs the stream.  Errors:
 * GI_ERR_INVALID_ARG (NULL), GI_ERR_CUDA. */
int gi_vset_size(gi_vset *s, int64_t *out, void *stream);

/* Which representations currently hold the set (a mask of GI_REP_*).
 * Errors: GI_ERR_INVALID_ARG (NULL). */
int gi_vset_reps(const gi_vset *s, uint32_t *reps);

/* Make the sparse representation valid (bitmap/bool -> ids, ascending order).
 * Errors: GI_ERR_INVALID_ARG (NULL), GI_ERR_OOM, GI_ERR_CUDA. */
int gi_vset_to_sparse(gi_vset *s, void *stream);

/* Make a dense representation valid: rep = GI_REP_BOOL or GI_REP_BITMAP.
 * Errors: GI_ERR_INVALID_ARG (NULL or another rep), GI_ERR_OOM, GI_ERR_CUDA. */
int gi_vset_to_dense(gi_vset *s, uint32_t rep, void *stream);

/*
 * Write the members in ascending order to dev_out (device, cap entries) and the
 * member count to *count (host).  Syncs the stream.  GI_ERR_INVALID_ARG if the set
 * has more than cap members (nothing is written then).
 */
int gi_vset_export(gi_vset *s, int32_t *dev_out, int64_t cap, int64_t *count, void *stream);

/* Replace the members by k device-resident ids (each in [0,n); duplicates removed).
 * Syncs the stream.  Errors: GI_ERR_INVALID_ARG (NULL, k < 0 or an id out of
 * range: the set is then left empty), GI_ERR_CUDA. */
int gi_vset_import(gi_vset *s, const int32_t *dev_ids, int64_t k, void *stream);

/* --------------------------------------------------------------- schedule -- */
/* configApplyDirection (Table 3) */
#define GI_DIR_SPARSE_PUSH 0  /* SparsePush                                   */
#define GI_DIR_DENSE_PUSH 1   /* DensePush                                    */
#define GI_DIR_DENSE_PULL 2   /* DensePull                                    */
#define GI_DIR_HYBRID_PULL 3  /* DensePull-SparsePush, chosen per iteration    */
#define GI_DIR_HYBRID_DPUSH 4 /* DensePush-SparsePush, chosen per iteration    */
#define GI_DIR_LEARNED 5      /* MLP picks SparsePush/DensePush/DensePull      */
#define GI_DIR_SPARSE_PULL 6  /* SparsePull: only the destinations of the `to` */
                              /* set pull, each over its in-edges (thread /   */
                              /* warp / block by degree); without a `to` set   */
                              /* and in the drivers it runs as DensePull      */

/* configApplyParallelization (Table 3) */
#define GI_BAL_VERTEX 0     /* vertex-parallel: one thread per vertex                     */
#define GI_BAL_EDGE_AWARE 1 /* edge-aware: thread / warp / CTA by degree (t_warp, t_cta)   */
#define GI_BAL_EDGE_PARALLEL 2 /* SparsePush one thread per arc (exclusive scan of the     */
                               /* frontier's degrees; each arc finds its source by binary  */
                               /* search); other traversals as EDGE_AWARE                  */

/* threshold rule used by the hybrid directions */
#define GI_RULE_BEAMER 0 /* push->pull when m_f > m_u/alpha; pull->push when |F| < n/beta */
#define GI_RULE_LIGRA 1  /* pull iff |F| + m_f > m/20                                     */

typedef struct gi_schedule {
  int32_t direction;    /* GI_DIR_*                                                  */
  uint32_t dense_rep;   /* frontier rep for dense traversals: GI_REP_BITMAP or BOOL  */
  int32_t balance;      /* GI_BAL_*                                                  */
  int32_t num_segments; /* SSG count for segmented pull (configApplyNumSSG); 1 = off  */
  int32_t block;        /* SparsePush block size: 128, 256 or 512 threads (the grid   */
                        /* keeps 2048 threads per SM); other kernels run 256          */
  int32_t t_warp;       /* edge-aware: degree >= t_warp goes to a warp                */
  int32_t t_cta;        /* edge-aware: degree >= t_cta goes to a whole block          */
  int32_t rule;         /* GI_RULE_*                                                 */
  float alpha, beta;    /* Beamer constants                                          */
  int32_t tile_edges;   /* pull tiles: arcs per tile (power of two, 256..8192; 256 =   */
                        /* one warp per tile, larger = one block per tile)            */
  int32_t t_heavy;      /* edge-aware push: degree >= t_heavy is split over all blocks */
  int32_t persistent;   /* gi_bfs / gi_sssp: 1 = run every level inside one cooperative */
                        /* persistent kernel (the batched engine's whole-GPU mode), the */
                        /* direction chosen on the device (LEARNED: the MLP; SPARSE_PUSH */
                        /* or DENSE_PUSH: push only; otherwise Beamer's rule); the trace */
                        /* then records only the level count.  2 = the level loop is a */
                        /* CUDA graph (a WHILE node over the library's per-level or    */
                        /* per-round kernels, direction and loop condition set on the  */
                        /* device, no host round trip per level; gi_sssp: see there),  */
                        /* built on first use and cached per graph and schedule;       */
                        /* trace: level count only.  0 = one host-driven round per level. */
  int32_t hot_cache;    /* PageRank / PageRankDelta / CC / SSSP DensePull over the whole */
                        /* graph (CC and SSSP: their driver rounds):                   */
                        /* the values of the (up to 24,576) highest-out-degree sources   */
                        /* are read from on-chip memory instead of one L2 sector per     */
                        /* arc (the GPU form of the cache partitioning of Sec. 2).       */
                        /* 1 = the hottest (up to 8,192) in shared memory, the rest in   */
                        /* L1, two persistent blocks per SM (tiles of                    */
                        /* 512..2048 arcs); 2 = a dense array cached in L1 (tiles of     */
                        /* 512..8192 arcs); 0 = off.  Results are bit-identical to 0.    */
                        /* Ignored elsewhere.  Built once per graph (4m bytes).          */
  int32_t seg_strategy; /* segmented pull (num_segments > 1): GI_SEG_FVC or GI_SEG_EVC    */
  int32_t delta;        /* gi_sssp only: 0 = Bellman-Ford in synchronous rounds (Sec. 7);  */
                        /* > 0 = delta-stepping with buckets of this width in weight units */
                        /* (see gi_sssp); same distances either way                        */
  int32_t dst_list;     /* gi_bfs (and gi_selector_profile's BFS) DensePull levels: 1 =    */
                        /* walk a compacted list of the unvisited vertices that have       */
                        /* in-arcs (the destination filter kept sparse: built once per     */
                        /* graph, 12 bytes per such vertex, shrunk at every pull level);   */
                        /* 0 = walk every vertex.  Same depths and parents either way.     */
} gi_schedule;

/* Defaults: HYBRID_PULL, BITMAP, EDGE_AWARE, 1 segment (FVC when segmented), 256
 * threads, t_warp 32, t_cta 256, Beamer alpha 14 beta 24, 2048-arc tiles, t_heavy 256,
 * not persistent, hot_cache 0, delta 0, dst_list 1.  Every driver rejects a schedule with a
 * field out of range with GI_ERR_INVALID_ARG. */
void gi_schedule_default(gi_schedule *s);

/* ------------------------------------------------------------ edgeset apply -- */
/*
 * Built-in edge functions (the `f` of apply/applyModified).  Each names the
 * vertex vectors it reads/writes through a kernel_args struct of device
 * pointers.  Push directions apply f with atomics, pull directions without
 * (dependence rules of Sec. 6).  All reductions are commutative and
 * associative or asyncMin, so any traversal order gives the same result
 * (integers bit-exact; float sums up to rounding order).
 */
#define GI_K_BFS 1   /* dstFilter depth[v]==-1; f: depth[v]=level, parent[v]=min(parent[v],u) */
#define GI_K_SSSP 2  /* f: dist[v] = min(dist[v], snap[u] + w(u,v))                         */
#define GI_K_CC 3    /* f: label[v] = min(label[v], snap[u])                                 */
#define GI_K_SUM 4   /* f: acc[v] += contrib[u]  (PageRank / PageRankDelta updateEdge)        */
#define GI_K_PROBE 5 /* f: count[v] += 1; srcsum[v] += u+1  (records the selected edges)      */

typedef struct { int32_t *depth; int32_t *parent; int32_t level; } gi_bfs_args;
/* parent may be NULL; otherwise unvisited entries must hold INT32_MAX on entry. */
typedef struct { int32_t *dist; const int32_t *snap; } gi_sssp_args;
/* snap[u] = dist of u at the start of the round, read for frontier sources only. */
typedef struct { int32_t *label; const int32_t *snap; } gi_cc_args;
typedef struct { const float *contrib; float *acc; } gi_sum_args;
typedef struct { int32_t *count; unsigned long long *srcsum; } gi_probe_args;

/* applyModified without deduplication (Table 2, disable_deduplication).  Honoured
 * for GI_K_BFS, whose function modifies each destination at most once; the other
 * kernels always deduplicate so the output never holds more than n entries. */
#define GI_NO_DEDUP 0x1u

/*
 * edges.from(from).to(to).srcFilter/dstFilter(kernel_id's filter).apply(f)
 * (out_modified == NULL) or .applyModified(f) (out_modified != NULL: receives
 * the destinations whose vector entry f changed, deduplicated unless
 * GI_NO_DEDUP).  from/to == NULL mean all vertices.  The traversal follows
 * sched->direction; hybrid and learned directions pick per call (this syncs
 * the stream to read the frontier statistics).  out_modified must not alias
 * from or to.  Errors: GI_ERR_INVALID_ARG, GI_ERR_UNSUPPORTED (pull direction
 * on a non-symmetric graph without gi_load_csc), GI_ERR_CUDA.
 */
int gi_edgeset_apply(gi_graph *g, gi_vset *from, gi_vset *to, const gi_schedule *sched, int32_t kernel_id,
                     const void *kernel_args, gi_vset *out_modified, uint32_t flags, void *stream);

/* ---------------------------------------------------------------- drivers -- */
/*
 * Per-iteration trace of a driver run (optional, host memory): for iteration i,
 * direction[i] (GI_DIR_SPARSE_PUSH/DENSE_PUSH/DENSE_PULL actually used),
 * frontier[i] = |F|, edges[i] = m_f (sum of out-degrees over F) and, if
 * features != NULL, the 16 selector features of the iteration at
 * features[16*i .. 16*i+15].  Any array pointer may be NULL.  Iterations past
 * `cap` run but are not recorded; `iterations` counts all of them.  For
 * delta-stepping SSSP an iteration is a relaxation round: F is the round's
 * sources, m_f the arcs of the class it relaxes, and phase[i] (may be NULL)
 * is 0 for a light round and 1 for a bucket's heavy round (0 elsewhere).
 */
typedef struct gi_trace {
  int32_t cap;        /* entries available in the arrays below                */
  int32_t iterations; /* filled in: number of iterations run                  */
  int32_t *direction;
  int64_t *frontier;
  int64_t *edges;
  float *features;
  int32_t *phase;
} gi_trace;

/*
 * Level-synchronous BFS from src (Sec. 7's BFS: SparsePush, DensePull with a
 * bitvector frontier and early exit, DensePush, or a hybrid).  depth_dev[n]:
 * hops from src, -1 if unreached.  parent_dev[n] (may be NULL): the smallest-id
 * in-neighbour one level closer to src (parent[src] = src, -1 if unreached);
 * the rule makes parents identical under every schedule.  Syncs the stream.
 * Errors: GI_ERR_INVALID_ARG (NULL, src out of range, bad schedule),
 * GI_ERR_UNSUPPORTED (DENSE_PULL without in-edges), GI_ERR_TIMEOUT (a level
 * cap or bounded wait of the persistent / graph-driven modes), GI_ERR_OOM,
 * GI_ERR_CUDA.
 */
int gi_bfs(gi_graph *g, int32_t src, int32_t *depth_dev, int32_t *parent_dev, const gi_schedule *sched,
           gi_trace *trace, void *stream);

/*
 * Single-source shortest paths from src on the graph's non-negative int32
 * weights; dist_dev[n]: the distance, INT32_MAX if unreachable (sums are
 * clamped at INT32_MAX).  Same distances under every schedule.
 * sched->delta == 0: frontier Bellman-Ford (Sec. 7's SSSP) in synchronous
 * rounds; round r relaxes the out-arcs of vertices whose distance dropped in
 * round r-1 using their start-of-round distance, in the direction the
 * schedule picks per round.
 * sched->delta > 0: delta-stepping (buckets of that width in weight units;
 * arcs lighter than delta are light): each bucket's light arcs are relaxed in
 * synchronous rounds until no distance in the bucket drops, then the heavy
 * arcs of the vertices settled in the bucket in one round, then the next
 * non-empty bucket.  Each round's direction (push over the round's sources, or
 * pull over every vertex's light or heavy in-arcs) is the schedule's; on a
 * directed graph delta-stepping rounds push (the arc classes are split from
 * the out-edges, once per graph and width, and cached).  The trace records
 * the counted rounds with their phase (0 light, 1 heavy).
 * sched->persistent: 0 = host-driven rounds; 1 = the batched engine's
 * whole-GPU persistent kernel (near/far rounds; trace: round count only);
 * 2 = the rounds as a CUDA graph (delta-stepping, or Bellman-Ford as one
 * bucket holding every arc), built on first use and cached per graph, width
 * and schedule; trace: round count only.  Syncs the stream.
 * Errors: GI_ERR_INVALID_ARG (NULL, no weights, src out of range, bad
 * schedule, a DENSE_PULL or HYBRID_PULL schedule on a directed graph loaded
 * without in-edge weights), GI_ERR_UNSUPPORTED (a forced pull direction
 * without in-edges), GI_ERR_TIMEOUT (a round cap or bounded wait of the
 * persistent / graph-driven modes), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_sssp(gi_graph *g, int32_t src, int32_t *dist_dev, const gi_schedule *sched, gi_trace *trace,
            void *stream);

/*
 * Builds ahead of the queries what a driver of `algo` (GI_ALGO_*) run with
 * `sched` would build on its first call on g (not in the paper; the results
 * of later calls do not change): the pull tiles of sched->tile_edges; for
 * GI_ALGO_SSSP with delta > 0 (or persistent == 2) the light / heavy arc split
 * and its pull views; for persistent == 2 the CUDA-graph level loop (BFS,
 * SSSP); for a host-driven GI_ALGO_BFS with dst_list the unvisited-list
 * storage.  Work is enqueued on `stream`, which is synchronized before the
 * return.  May run in another host thread while queries run on other
 * graphs.  Errors: GI_ERR_INVALID_ARG (NULL, unknown algo, bad schedule,
 * SSSP without weights), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_prepare(gi_graph *g, int32_t algo, const gi_schedule *sched, void *stream);

/*
 * Connected components by synchronous min-label propagation (Sec. 7's CC):
 * label_dev[n] = smallest vertex id of v's component (symmetric graphs).
 * Syncs the stream.  Errors: GI_ERR_INVALID_ARG, GI_ERR_UNSUPPORTED (DENSE_PULL
 * without in-edges), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_cc(gi_graph *g, int32_t *label_dev, const gi_schedule *sched, gi_trace *trace, void *stream);

/*
 * PageRank (Sec. 7's PR): iters power iterations of
 * PR[v] = (1-d)/n + d * sum_{u in in(v)} PR[u]/outdeg(u) from PR = 1/n in FP32
 * (FP32 accumulation), then division by the FP64 sum of all ranks.
 * sched->direction: DENSE_PULL (default; segmented when num_segments > 1) or
 * DENSE_PUSH.  rank_dev[n] receives the normalised ranks.  Syncs the stream.
 * Errors: GI_ERR_INVALID_ARG (NULL, iters < 0, damping outside [0,1]),
 * GI_ERR_UNSUPPORTED (pull without in-edges), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_pagerank(gi_graph *g, float damping, int32_t iters, float *rank_dev, const gi_schedule *sched,
                void *stream);

/*
 * PageRank without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not allocate GPU memory once they are
 * running -- for example code that works inside a fixed, pre-reserved memory
 * budget, or a plug-in whose host application owns the device heap through its
 * own allocator -- and so cannot use gi_load_csr / gi_pagerank, which allocate
 * the graph copy, tiles and working vectors.
 *
 * Same result as gi_pagerank (the power iteration described there, FP32 with
 * an FP64 normalisation) on CSR arrays the caller already holds on the device:
 * in_offsets[n+1] / in_indices[m] are the in-edges (for a symmetric graph, the
 * CSR itself); out_offsets[n+1] gives out-degrees (NULL: use in_offsets, i.e.
 * the graph is symmetric).  rank[n] (device) receives the normalised ranks.
 * The caller owns every array; the library only reads the inputs and writes rank.
 *
 * Working memory is a file-scope device array sized for GI_STATIC_PR_MAX_N
 * vertices (two float vectors plus 1024 doubles, about 8 MB); every GPU that
 * loads the library holds it until the process exits.  Larger graphs are
 * rejected with GI_ERR_INVALID_ARG before any work is queued.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  Under lazy
 * module loading (the CUDA default) the driver reserves the array when that
 * first call loads the library's module on the device, so the first call may
 * itself need the ~8 MB: make it during set-up, while memory is still
 * available, and every later call reuses the array.  All calls
 * share the one array and the kernels re-initialise what they read, so
 * results do not depend on earlier calls -- but calls whose work overlaps on
 * the GPU (different streams, or host threads) race on the array and must be
 * serialised by the caller.  Errors: GI_ERR_INVALID_ARG (sizes, NULL pointers,
 * n > GI_STATIC_PR_MAX_N), GI_ERR_UNSUPPORTED (m >= 2^31), GI_ERR_CUDA.
 */
#define GI_STATIC_PR_MAX_N (1 << 20)
int gi_pagerank_static(const int32_t *in_offsets, const int32_t *in_indices, const int32_t *out_offsets, int64_t n,
                       int64_t m, float damping, int32_t iters, float *rank, void *stream);

/*
 * PageRankDelta (Fig. 1, with the round-1 update order of the GraphIt program
 * of Fig. 3): Rank = 0, Delta = 1/n, all vertices active; each round the active
 * vertices propagate Delta/outdeg, every vertex updates Delta and Rank, and
 * those with |Delta| > eps*Rank stay active.  iters rounds, FP32.  rank_dev[n]
 * receives Rank (not normalised).  The edge traversal per round follows sched
 * (hybrid by default: DensePull when the active set is large, SparsePush else).
 * Syncs the stream.  Errors: GI_ERR_INVALID_ARG (NULL, iters < 0, eps < 0),
 * GI_ERR_UNSUPPORTED (DENSE_PULL without in-edges), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_pagerank_delta(gi_graph *g, float damping, float eps, int32_t iters, float *rank_dev,
                      const gi_schedule *sched, gi_trace *trace, void *stream);

/*
 * Betweenness Centrality from one source (Sec. 7 runs BC from single starting
 * points, synchronously, as two edgeset applies per level).  Brandes'
 * single-source dependencies:
 *   sigma[v] = number of shortest src-v paths (forward apply s1, level by
 *              level; sigma[src] = 1);
 *   delta[u] = sum over out-arcs (u,v) with d(v) = d(u)+1 of
 *              sigma[u] / sigma[v] * (1 + delta[v])  (backward apply s2).
 * dependency_dev[n] (device, FP64) receives delta (0 at src and at unreached
 * vertices); with accumulate != 0 it is added to what the array holds, so
 * summing calls over all sources gives BC.  sigma_dev[n] (FP64, may be NULL)
 * receives sigma (exact integers below 2^53).  s1 follows sched->direction
 * like gi_bfs; s2 runs a SparsePull over each level's vertices along their
 * out-edges (t_warp, t_cta), or, on symmetric graphs, the tiled pull over all
 * rows when sched->direction is DENSE_PULL or, for hybrid and learned
 * directions, when the level's |F| + m_f exceeds m/20; push directions and
 * SPARSE_PULL keep the SparsePull.
 * Trace: the forward levels.  Errors: GI_ERR_INVALID_ARG, GI_ERR_UNSUPPORTED
 * (DENSE_PULL without in-edges), GI_ERR_OOM, GI_ERR_CUDA.  Syncs the stream.
 */
int gi_bc(gi_graph *g, int32_t src, double *dependency_dev, double *sigma_dev, int32_t accumulate,
          const gi_schedule *sched, gi_trace *trace, void *stream);

/* ------------------------------------------------------------ selector -- */
/*
 * Load the learned direction selector: a 16-64-64-3 ReLU perceptron, params as
 * float32 W1[64][16], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] (host memory,
 * `count` = 5443 floats), plus feature normalisation mean[16] and inv_std[16].
 * Used by GI_DIR_LEARNED: the network picks the argmin of its predicted
 * log-times for a frontier with |F| + m_f >= m / 200; a smaller frontier is
 * pushed (SparsePush) without an evaluation.  Until loaded, LEARNED falls back
 * to the Beamer rule.
 * Errors: GI_ERR_INVALID_ARG (NULL or count != 5443), GI_ERR_CUDA.
 */
int gi_selector_load(const float *params, int32_t count, const float *mean, const float *inv_std);

/* Number of parameters of the selector network (5443; never fails). */
int gi_selector_num_params(void);

/*
 * Training of the selector on the GPU (not in the paper).  All pointers are
 * device memory, float32.  params: the 5443 parameters in the layout of
 * gi_selector_load; X[B][16] features, T[B][3] targets (log-time of
 * SparsePush, DensePush, DensePull), M[B][3] mask (1 = target measured).
 * gi_mlp_loss_grad writes grad[5443] (overwritten) and loss[2] = {masked MSE
 * sum_{b,j} M (Y-T)^2 / sum M, sum M}.  gi_mlp_forward writes Y[B][3].
 * gi_mlp_adam applies one Adam step (Kingma & Ba) with step number t >= 1,
 * updating params and the moment vectors m, v in place.  Asynchronous on
 * `stream`.  Errors: GI_ERR_INVALID_ARG (NULL, B < 1, t < 1), GI_ERR_OOM,
 * GI_ERR_CUDA.
 */
int gi_mlp_loss_grad(const float *params, const float *X, const float *T, const float *M, int64_t B, float *grad,
                     float *loss, void *stream);
int gi_mlp_forward(const float *params, const float *X, int64_t B, float *Y, void *stream);
int gi_mlp_adam(float *params, const float *grad, float *m, float *v, int32_t t, float lr, float b1, float b2,
                float eps, void *stream);

/*
 * Training data for the selector (not in the paper): run BFS (GI_K_BFS) or
 * SSSP (GI_K_SSSP) from src; at every level keep the state, run SparsePush,
 * DensePush and DensePull from it, each timed with CUDA events on `stream`,
 * and continue from the common result.  For level i < cap, features[16*i..]
 * (host) receive the level's 16 selector features and times_ms[3*i..] (host)
 * the three durations in milliseconds; *levels the number of levels recorded.
 * With sched->delta > 0 (GI_K_SSSP, symmetric graphs): the counted
 * delta-stepping rounds, SparsePush and DensePull over the round's arc class
 * timed (DensePush is not offered: its time is -1).  BFS pulls follow
 * sched->dst_list.  Syncs the stream.  Needs the in-edges (symmetric graph or
 * gi_load_csc).
 * Errors: GI_ERR_INVALID_ARG (NULL, other kernel_id, src out of range, cap < 0),
 * GI_ERR_UNSUPPORTED (no in-edges; delta-stepping on a directed graph),
 * GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_selector_profile(gi_graph *g, int32_t kernel_id, int32_t src, const gi_schedule *sched, int32_t cap,
                        float *features, float *times_ms, int32_t *levels, void *stream);

/* ---------------------------------------------------------------- batched -- */
/*
 * Many BFS / SSSP queries over several graphs in one persistent launch (not in
 * the paper, which runs one query at a time).  The launch is a grid of
 * thread-block clusters; each cluster claims the next query from a global
 * counter and runs it to completion with cluster barriers between levels
 * (BFS: SparsePush or early-exit DensePull per level; SSSP: Bellman-Ford push
 * with asynchronous min updates, i.e. the asyncMin of Sec. 6 -- same final
 * distances as gi_sssp, different round counts).  No cluster ever waits for
 * another.
 */
typedef struct gi_batch_opts {
  int32_t cluster_size; /* CTAs per query: 1, 2, 4 or 8 (default 4); 0 = whole GPU: every  */
                        /* co-resident block (cooperative launch) works on one query at a */
                        /* time, levels separated by a software grid barrier whose wait   */
                        /* gives up after ~2 s with GI_ERR_TIMEOUT                         */
  int32_t clusters;     /* clusters launched; 0 = SM count / cluster_size                  */
  int32_t selector;     /* BFS direction per level: GI_DIR_SPARSE_PUSH (always push),      */
                        /* GI_DIR_HYBRID_PULL (Beamer rule) or GI_DIR_LEARNED (the MLP)    */
  float alpha, beta;    /* Beamer constants                                                */
  int64_t level_cap;    /* give up after this many levels (0 = 4n+16): GI_ERR_TIMEOUT     */
  int32_t *levels;      /* host, n_q entries or NULL: levels (BFS) / rounds (SSSP) run     */
  float sssp_delta;     /* SSSP threshold step = sssp_delta x mean arc weight (0: 2.0;     */
                        /* < 0: no threshold, every frontier source relaxed each round)    */
  int32_t order;        /* order in which clusters claim queries: 0 = as given, 1 =        */
                        /* largest graph first, SSSP before BFS (shorter makespan)          */
  int32_t t_warp;       /* expansion bins: frontier sources with >= t_warp arcs are spread */
                        /* over a warp (1..32; 0 = 32) ...                                 */
  int32_t t_cta;        /* ... and with >= t_cta arcs over the CTA (>= t_warp; 0 = 1024)   */
  int32_t *const *parents; /* host array of n_q device pointers, or NULL: a BFS query whose */
                        /* entry is non-NULL also receives the canonical parents there (n   */
                        /* of its graph entries; as gi_bfs: parent[src] = src, -1 if        */
                        /* unreached); entries of SSSP queries are ignored                  */
} gi_batch_opts;

/* Defaults: cluster_size 4, clusters 0, HYBRID_PULL, alpha 14, beta 24, level_cap 0,
 * levels NULL, sssp_delta 0, order 1, t_warp 32, t_cta 1024, parents NULL (never fails). */
void gi_batch_opts_default(gi_batch_opts *o);

/*
 * graphs[n_graphs]: loaded graphs.  Query i (host arrays): graph q_graph[i],
 * source q_src[i], algorithm q_algo[i] (GI_ALGO_BFS or GI_ALGO_SSSP); its
 * result goes to out_dev[i] (a device pointer with n of that graph entries:
 * BFS depth, -1 if unreached; SSSP distance, INT32_MAX if unreachable --
 * the same values as gi_bfs / gi_sssp).  q_ns[n_q] (host, may be NULL)
 * receives each query's device time in nanoseconds (%globaltimer).  opts may
 * be NULL (defaults).  Syncs the stream.  Errors: GI_ERR_INVALID_ARG,
 * GI_ERR_TIMEOUT (a query hit level_cap), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_batch_run(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph, const int32_t *q_src,
                 const int32_t *q_algo, int32_t n_q, int32_t *const *out_dev, int64_t *q_ns,
                 const gi_batch_opts *opts, void *stream);

/*
 * The same in three steps, so that the launch can be captured in a CUDA graph
 * and replayed: gi_batch_plan_create validates the queries, allocates the
 * working memory and uploads the query tables (syncs the stream);
 * gi_batch_plan_launch enqueues one memset and the single persistent kernel
 * on `stream` (no allocation, no host synchronisation: capturable);
 * gi_batch_plan_results copies per-query times and level counts (either may be
 * NULL) and reports GI_ERR_TIMEOUT if a query hit the level cap (syncs);
 * gi_batch_plan_free releases everything (NULL is a no-op).  Outputs go to the
 * out_dev pointers given at creation, which must stay valid while the plan is
 * used.  Errors: as gi_batch_run (create), GI_ERR_INVALID_ARG (NULL plan),
 * GI_ERR_TIMEOUT and GI_ERR_CUDA (results).
 */
typedef struct gi_batch_plan gi_batch_plan;
int gi_batch_plan_create(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph, const int32_t *q_src,
                         const int32_t *q_algo, int32_t n_q, int32_t *const *out_dev, const gi_batch_opts *opts,
                         void *stream, gi_batch_plan **out);
int gi_batch_plan_launch(gi_batch_plan *p, void *stream);
int gi_batch_plan_results(gi_batch_plan *p, int64_t *q_ns, int32_t *levels, void *stream);
int gi_batch_plan_free(gi_batch_plan *p);

/* ------------------------------------------------------------- autotuner -- */
/* algorithms the autotuner runs (the drivers above with their Sec. 7 settings) */
#define GI_ALGO_BFS 1            /* gi_bfs from src, depths only          */
#define GI_ALGO_SSSP 2           /* gi_sssp from src                      */
#define GI_ALGO_CC 3             /* gi_cc                                 */
#define GI_ALGO_PAGERANK 4       /* gi_pagerank, damping 0.85, 20 iters   */
#define GI_ALGO_PAGERANK_DELTA 5 /* gi_pagerank_delta, 0.85, 1e-7, 10     */

/*
 * Schedule autotuner (the paper tunes schedules with OpenTuner, Sec. 6): keeps
 * start->direction/balance/rule and searches tile_edges, t_warp, t_cta,
 * t_heavy, block, hot_cache (not BFS), the dense frontier representation
 * dense_rep (not PageRank), num_segments and seg_strategy (PageRank
 * DensePull), delta (SSSP: Bellman-Ford or delta-stepping bucket widths),
 * dst_list (BFS) and, for rule-based BFS hybrids, Beamer's alpha/beta: random
 * candidates for the
 * first third of `budget`
 * trials, then a coordinate sweep around the best (one knob at a time, each
 * of its other values in turn, then the next knob).  Each candidate runs once to
 * warm up and is timed (best of 2) with CUDA events on `stream`; a candidate
 * whose output differs from start's (integers bit-exact, ranks beyond 1e-4
 * relative) is rejected.  *best receives the fastest valid schedule, *best_ms
 * and *start_ms (may be NULL) its time and start's.  Syncs the stream.
 * Errors: GI_ERR_INVALID_ARG (NULL, unknown algo, budget outside [1, 100000],
 * src out of range, SSSP without weights), GI_ERR_OOM, GI_ERR_CUDA, or a
 * driver's error for a candidate.
 */
int gi_autotune(gi_graph *g, int32_t algo, int32_t src, const gi_schedule *start, int32_t budget, uint64_t seed,
                gi_schedule *best, double *best_ms, double *start_ms, void *stream);

/*
 * Autotuner of the batched engine (the same search applied to the batched
 * launch, not in the paper): keeps start's selector and Beamer constants and
 * searches cluster_size (1, 2, 4, 8), the expansion bins t_warp (8, 16, 32)
 * and t_cta (128 .. 4096), sssp_delta (0.5 .. 8) and the claim order, each
 * candidate a plan over the given queries (gi_batch_plan_create) whose
 * launch is timed with CUDA events on `stream` (best of two after a
 * warm-up); a candidate whose results differ from start's in any query is
 * rejected.  start may be NULL (defaults); its levels and parents pointers are
 * not used while tuning and are copied to *best.  The library allocates the
 * output buffers of the candidates (the sum of the queried graphs' vertex
 * counts, twice).  Syncs the stream.  Errors: as gi_batch_plan_create,
 * GI_ERR_INVALID_ARG (budget outside [1, 100000]), GI_ERR_OOM, GI_ERR_CUDA.
 */
int gi_batch_autotune(gi_graph *const *graphs, int32_t n_graphs, const int32_t *q_graph, const int32_t *q_src,
                      const int32_t *q_algo, int32_t n_q, const gi_batch_opts *start, int32_t budget, uint64_t seed,
                      gi_batch_opts *best, double *best_ms, double *start_ms, void *stream);

/* -------------------------------------------------------------- profiling -- */
/*
 * Host-side instrumentation for benchmarks (not part of the paper).  The
 * library counts every kernel it launches.  With timing on, each launch of the
 * timed kernel classes below is bracketed by CUDA events recorded on the
 * launching stream.  Process-wide state; not meant for concurrent callers.
 */
#define GI_KCLASS_PR_PULL 0    /* tiled DensePull of PageRank (vertex update fused)        */
#define GI_KCLASS_PRD_PULL 1   /* tiled DensePull of PageRankDelta (vertex filter fused)   */
#define GI_KCLASS_MIN_PULL 2   /* tiled DensePull of CC / SSSP (min reduction)             */
#define GI_KCLASS_PUSH 3       /* SparsePush / DensePush expansion                         */
#define GI_KCLASS_BFS_PULL 4   /* early-exit BFS DensePull                                 */
#define GI_KCLASS_OTHER_PULL 5 /* other tiled pulls (sum, probe, segments)                 */
#define GI_KCLASS_BATCH 6      /* the batched persistent engine                            */

/* Turn per-launch event timing on (1) or off (0); counting is always on (never fails). */
int gi_stats_enable(int timing_on);
/* Zero the launch counter and drop recorded timings (never fails). */
int gi_stats_reset(void);
/*
 * Launches since the last reset (*launches), and for kernel class `kclass`
 * (-1 = all timed classes) the number of timed launches and their summed
 * device time in milliseconds.  Waits for the recorded events.  Errors:
 * GI_ERR_INVALID_ARG (unknown class), GI_ERR_CUDA.
 */
int gi_stats_read(int32_t kclass, int64_t *launches, int64_t *timed_launches, double *timed_ms);

/*
 * Instrumentation (not in the paper): *arcs = the arcs that the block-tiled
 * DensePulls on g gathered (staged for reduction) while per-launch timing
 * was on, since the last reset -- every arc of a short tile, the arcs of a
 * long row only when its destination passes the filters; warp tiles and the
 * vertex-parallel pull are not counted.  reset != 0 zeroes the count after
 * reading it.  Synchronizes the device.  Errors: GI_ERR_INVALID_ARG (NULL),
 * GI_ERR_CUDA.
 */
int gi_stats_pull_arcs(gi_graph *g, int32_t reset, int64_t *arcs);

/*
 * Gather ceiling (instrumentation, not in the paper): one launch on `stream`
 * that streams idx[m] (device, 16-byte aligned; every id in [0, n)) with
 * 16-byte loads and reads table[idx[i]] (device, n floats) for every i --
 * the two memory streams of a dense pull with nothing else -- so m divided
 * by its CUDA-event time bounds the rate at which any pull over the same
 * source ids can gather.  out (device, one float) is written only to keep the
 * loads from being removed.  Errors: GI_ERR_INVALID_ARG, GI_ERR_CUDA.
 */
int gi_gather_rate(const int32_t *idx, int64_t m, const float *table, int64_t n, float *out, void *stream);

/* ------------------------------------------------------- fault injection -- */
/*
 * Test hooks (host-side, process-wide; not in the paper).  After n more
 * successful device allocations, every allocation the library attempts fails
 * and the call returns GI_ERR_OOM (n < 0 turns the hook off).  Every call must
 * release what it allocated on such a failure; gi_debug_pool_used reports the
 * bytes currently allocated from the device's default pool, which the library
 * allocates from, so a test can check that nothing leaked.
 */
int gi_debug_fail_allocs_after(int64_t n);
int gi_debug_pool_used(int64_t *bytes);
/*
 * The grid barrier of the whole-GPU persistent mode (gi_batch_opts.cluster_size
 * = 0) waits for k more arrivals than there are blocks, so its bounded wait
 * (about 2 s) runs out: the kernel then stops and the call returns
 * GI_ERR_TIMEOUT with the context intact.  k = 0 restores normal operation.
 */
int gi_debug_barrier_phantoms(int32_t k);

#ifdef __cplusplus
}
#endif
#endif /* GRAPHIT_GB_H */
