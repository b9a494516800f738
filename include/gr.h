/*
 * gr — frontier-operator graph primitives for one GB300 (sm_103a).
 *
 * A C ABI over hand-written CUDA kernels implementing the data-centric
 * frontier model of Wang et al., "Gunrock: A High-Performance Graph
 * Processing Library on the GPU" (PPoPP'16): the advance, filter and
 * direction-optimising pull operators (Sec. 4.1, 4.4, 4.5) and the five
 * primitives built on them (Sec. 5): BFS, SSSP, BC, CC and PageRank.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Graph: CSR as in Sec. 3 — row offsets R (int32, n+1 entries, R[0] = 0,
 *   non-decreasing, R[n] = m) and column indices C (int32, m entries, each
 *   in [0, n)), optional per-edge weights W (uint32, m entries). Undirected
 *   graphs are given symmetrised (both (u,v) and (v,u) stored), as the paper
 *   converts all its datasets (Sec. 6). Self-loops and duplicate entries are
 *   accepted. m must not exceed INT32_MAX.
 * Output pointers: device memory or page-locked host memory of the stated
 *   length, owned by the caller. Host outputs are filled by a copy at the
 *   end of the call's work on `stream`; device outputs are written in stream
 *   order. A call returns once its work is enqueued, except where a
 *   "(host)" scalar output forces a stream synchronisation.
 * stream: a cudaStream_t passed as void*; NULL is the legacy default stream.
 * Concurrency: calls on one gr_graph share its scratch memory; the library
 *   orders them on the device (a later call on another stream waits for the
 *   earlier one). Independent concurrent queries go through gr_server.
 * Errors: every call returns a gr_status; nothing is thrown across the ABI.
 *   GR_EINVAL for bad arguments (checked before any device work),
 *   GR_ENOMEM when device allocation fails, GR_ECUDA for other CUDA errors,
 *   GR_ETIMEOUT when a bounded device-side wait gave up (the graph stays
 *   usable). gr_last_error() returns this thread's last message.
 */
#ifndef GR_H
#define GR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gr_status {
  GR_OK = 0,
  GR_EINVAL = 1,
  GR_ENOMEM = 2,
  GR_ECUDA = 3,
  GR_ETIMEOUT = 4,
  GR_EBUSY = 5
} gr_status;

/* Opaque graph handle: owns device copies of R, C, W, derived per-graph data
 * (degree statistics, isolated-vertex bitmap, symmetry flag) and scratch. */
typedef struct gr_graph gr_graph;

/* Traversal direction policy (Sec. 4.5 "Push vs. pull traversal"). */
enum {
  GR_DIR_AUTO = 0, /* tuned push<->pull switching (needs a symmetric graph) */
  GR_DIR_PUSH = 1, /* push (top-down) advance on every level */
  GR_DIR_PULL = 2  /* push on the source's level, pull on every later level */
};

/* Level-loop driver. */
enum {
  GR_MODE_AUTO = 0,       /* chosen by the tuner from the graph's shape */
  GR_MODE_LAUNCH = 1,     /* host enqueues batches of level kernels that
                             exit early once the traversal is done */
  GR_MODE_GRAPH = 2,      /* one CUDA graph whose device-side while loop
                             runs one level per iteration */
  GR_MODE_PERSISTENT = 3  /* one cooperative kernel runs every level with a
                             bounded-spin grid barrier between levels; for a
                             BFS on a graph of maximum degree <= 16 one
                             thread-block cluster runs the levels first and
                             hands a frontier of more than 32768 vertices to
                             that kernel */
};

/* Options; pass NULL for tuned defaults. Zero in a field means "tuned". */
typedef struct gr_opts {
  int32_t direction;  /* GR_DIR_* */
  int32_t mode;       /* GR_MODE_* */
  int32_t block;      /* persistent BFS: blocks per SM (0: tuned) */
  int32_t chunk;      /* merge-path items per block chunk (0: tuned) */
  float alpha;        /* push->pull when frontier edges > unexplored/alpha */
  float beta;         /* pull->push when frontier vertices < n/beta */
  uint32_t delta;     /* SSSP near/far bucket width (0: tuned,
                         UINT32_MAX: no split, one bucket) */
  int32_t max_iters;  /* cap on device-side iterations (0: default) */
} gr_opts;

/* Create a graph from a CSR (Sec. 3; Alg. 1 operates on such a graph).
 * n >= 1 vertices, m >= 0 entries. row_off[n+1], col[m] and, if not NULL,
 * w[m] are host pointers when inputs_on_device == 0 and device pointers
 * otherwise; they are validated, copied and not retained. On success *out
 * holds a new handle to release with gr_graph_destroy. */
gr_status gr_graph_create(int32_t n, int64_t m, const int32_t *row_off,
                          const int32_t *col, const uint32_t *w,
                          int inputs_on_device, void *stream, gr_graph **out);

/* Release a graph and all device memory it owns (synchronises its work). */
gr_status gr_graph_destroy(gr_graph *g);

/* Per-graph statistics computed at creation (host scalars; any may be NULL):
 * vertex count, entry count, maximum degree, number of degree-0 vertices,
 * whether the CSR is symmetric (every (u,v) has a (v,u)), and whether
 * weights are present. */
gr_status gr_graph_info(const gr_graph *g, int32_t *n, int64_t *m,
                        int32_t *max_degree, int32_t *num_isolated,
                        int32_t *symmetric, int32_t *has_weights);

/* Breadth-first search from src (Sec. 5.1): depth[n] (int32) receives the
 * hop count from src, -1 where unreached; parent[n] (int32, may be NULL)
 * receives a valid BFS parent of each reached vertex (parent[src] = src),
 * -1 where unreached. Depth is unique; the parent is any vertex one level up
 * that has an edge to the child. Push levels run the load-balanced advance
 * (Sec. 4.4) fused with the visited-bitmap filter (Sec. 4.1, 4.5
 * "Idempotent vs. non-idempotent"); pull levels run the bitmap pull advance
 * (Sec. 4.5). */
gr_status gr_bfs(gr_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                 const gr_opts *opts, void *stream);

/* k breadth-first searches, one after another, each exactly as gr_bfs
 * (Sec. 5.1) from srcs[i] into depth[i][n] and, when parent is not NULL and
 * parent[i] is not NULL, parent[i][n]. srcs (k entries), depth and parent
 * (k pointers each) are host arrays; each output pointer is host or device
 * memory, as for gr_bfs. Results bound for host memory are copied out on a
 * copy stream of the graph while the next search runs, through two device
 * staging sets that alternate between searches (4n bytes per output each,
 * allocated at first use and kept by the graph). With page-locked host
 * outputs the copies overlap the searches; with pageable ones each copy
 * completes before the next search is enqueued. When `stream` reaches the
 * end of the call's work, every output, host or device, is complete.
 * k = 0 does nothing. Every source and output pointer is checked before
 * any work is enqueued (GR_EINVAL). */
gr_status gr_bfs_multi(gr_graph *g, int32_t k, const int32_t *srcs, int32_t *const *depth,
                       int32_t *const *parent, const gr_opts *opts, void *stream);

/* Number of levels (including the source's) and of pull levels of the last
 * completed gr_bfs on this graph (host scalars; synchronises). */
gr_status gr_bfs_stats(gr_graph *g, int32_t *levels, int32_t *pull_levels);

/* Single-source shortest paths from src over non-negative integer weights
 * (Alg. 1; Sec. 4.5 "Priority Queue"; Sec. 5.2). Requires weights.
 * dist[n] (uint32) receives the shortest distance, 0xFFFFFFFF where
 * unreachable (sums that do not fit below 0xFFFFFFFF count as unreachable);
 * pred[n] (int32, may be NULL) receives, for each reached v != src, the
 * smallest u with an edge (u, v) and dist[u] + w(u, v) = dist[v];
 * pred[src] = src; -1 where unreachable (with zero-weight edges pred may
 * contain cycles among equal-distance vertices). opts->delta sets the
 * near/far bucket width (0: tuned, UINT32_MAX: a single bucket); the
 * distances do not depend on it. Direction (the pull form of Sec. 4.5
 * applied to the relaxation, which the paper leaves to future work): on a
 * symmetric CSR a relaxation whose near frontier holds at least m /
 * opts->alpha edges (opts->alpha 0: the tuned threshold, by default never)
 * runs as a pull, every vertex taking the minimum over its in-edges;
 * opts->direction GR_DIR_PUSH never pulls, GR_DIR_PULL (symmetric CSR
 * only, else GR_EINVAL) pulls every relaxation. Distances do not depend on
 * the direction. */
gr_status gr_sssp(gr_graph *g, int32_t src, uint32_t *dist, int32_t *pred,
                  const gr_opts *opts, void *stream);

/* k single-source shortest-path searches in one run (Alg. 1; Sec. 4.5
 * "Priority Queue"; Sec. 5.2), from the host array srcs[k] (repeats
 * allowed) into dist[k*n] (uint32, device or host memory, source-major:
 * dist[i*n + v] is the distance from srcs[i] to v), each equal to gr_sssp's
 * dist for that source. The k searches run as one near/far search over k
 * disjoint copies of the graph (vertex i*n + v is v in copy i, which holds
 * source i only), so they share the device-side loop: on high-diameter
 * graphs, where an iteration costs a grid barrier rather than bandwidth, k
 * searches take about the time of one. No pred output. 1 <= k <= 64 with
 * k*n + 2 and k*m at most INT32_MAX, else GR_EINVAL (the message states the
 * graph's limit); requires weights. opts->mode GR_MODE_PERSISTENT runs the
 * cooperative kernel; GR_MODE_GRAPH is taken as GR_MODE_LAUNCH (host-driven
 * batches of iteration kernels). Scratch grows with k: about 32*k*n bytes,
 * kept by the graph for the next call. */
gr_status gr_sssp_batch(gr_graph *g, const int32_t *srcs, int32_t k, uint32_t *dist,
                        const gr_opts *opts, void *stream);

/* gr_sssp_stats for the last completed gr_sssp_batch on this graph. */
gr_status gr_sssp_batch_stats(gr_graph *g, int32_t *iterations, int32_t *phases,
                              int64_t *relaxations);

/* Statistics of the last completed gr_sssp on this graph (host scalars;
 * synchronises): device-loop iterations, near/far phases (splits) and
 * edges expanded. Returns GR_ETIMEOUT if that run hit its iteration cap
 * (opts->max_iters) or a device-side wait limit. */
gr_status gr_sssp_stats(gr_graph *g, int32_t *iterations, int32_t *phases,
                        int64_t *relaxations);

/* Relaxations of the last completed gr_sssp on this graph that ran in pull
 * form (host scalar; synchronises). */
gr_status gr_sssp_pull_stats(gr_graph *g, int32_t *pulls);

/* Connected components (Sec. 5.4): label[n] (int32) receives, for every
 * vertex, the smallest vertex id of its component (weakly connected
 * components for a directed CSR). *num_components (host, may be NULL)
 * receives the number of components; asking for it synchronises. Hooking
 * links the larger root under the smaller over the edge frontier, pointer
 * jumping then points every vertex at its root. On a symmetric CSR the
 * hooking pass is sampled: every vertex first hooks to its first two
 * neighbours, the trees are compressed, and only the vertices outside the
 * component most of a fixed sample of vertices falls in hook all their
 * edges (the labels are the same; the call synchronises once to read the
 * sample). opts is unused. */
gr_status gr_cc(gr_graph *g, int32_t *label, int32_t *num_components,
                const gr_opts *opts, void *stream);

/* PageRank (Sec. 5.5), pull form, FP32 ranks with FP64 reductions:
 * r'[v] = (1 - damping)/n + damping * (sum over edges (u, v) of
 * r[u]/deg(u) + D/n), D = sum of r[u] over vertices of out-degree 0,
 * starting from r = 1/n. Stops after max_iter iterations or once
 * sum |r' - r| < tol. rank[n] (float) receives the ranks; *iters (host, may
 * be NULL) the iterations run (asking for it synchronises). damping must lie
 * in (0, 1), max_iter >= 0, tol >= 0. A directed CSR is transposed once on
 * the device for the in-neighbour gather. opts->mode GR_MODE_LAUNCH runs
 * host-driven batches instead of the device-side loop. */
gr_status gr_pagerank(gr_graph *g, float damping, int32_t max_iter, double tol,
                      float *rank, int32_t *iters, const gr_opts *opts,
                      void *stream);

/* Batched BFS from k in [1, 64] sources at once (one bit lane per source).
 * A level whose frontier (over all lanes) has fewer than m/16 edges pushes
 * the lanes of the frontier's vertices to their neighbours; the others pull
 * over every vertex, reading each column index once for all lanes. Pulls
 * need in-neighbours = out-neighbours, so on a directed (non-symmetric) CSR
 * every level pushes (along out-edges, as gr_bfs traverses). srcs[k]
 * is a host array of vertices (repeats allowed). depth[k*n] (int32) receives
 * source-major results: depth[i*n + v] is the hop count from srcs[i] to v,
 * -1 where unreached, equal to gr_bfs's depth for that source. The whole
 * level loop is one cooperative kernel (a bounded grid barrier per level,
 * directions decided on the device): the call enqueues its work and returns
 * without synchronising. opts->max_iters > 0 caps the levels; a traversal
 * stopped by that cap or by a barrier wait that ran out is reported by
 * gr_bfs_batch_stats. */
gr_status gr_bfs_batch(gr_graph *g, const int32_t *srcs, int32_t k,
                       int32_t *depth, const gr_opts *opts, void *stream);

/* Levels of the last gr_bfs_batch on g (host output; synchronises):
 * *levels = 1 + the largest depth reached over all lanes. GR_ETIMEOUT if
 * that traversal stopped at a device-side limit (its depths are then
 * incomplete). */
gr_status gr_bfs_batch_stats(gr_graph *g, int32_t *levels);

/* Betweenness centrality (Brandes; Sec. 5.3): bc[n] (double) receives
 * bc[v] = sum over s in srcs, t != s of sigma_st(v) / sigma_st, v not in
 * {s, t}, where sigma_st counts shortest (unweighted) s-t paths: no halving
 * for undirected graphs, no normalisation; on a directed CSR paths follow
 * out-edges. srcs[k] is a host array (k >= 0, repeats counted). Sources run
 * in batches of 64 bit lanes (the levels as gr_bfs_batch runs them); path
 * counts are exact uint64 integers, and a batch whose counts pass 2^64 - 1
 * is counted again in FP64; dependencies are FP64. Returns GR_EINVAL if a
 * path count overflows FP64 (e.g. large grids). The forward levels of a
 * batch run in one cooperative kernel that keeps every level's lane masks;
 * it stops when it needs more mask arrays than are allocated, and the call
 * allocates more and resumes it. The call synchronises after each batch's
 * forward pass (for its level count) and at the end. */
gr_status gr_bc(gr_graph *g, const int32_t *srcs, int32_t k, double *bc,
                const gr_opts *opts, void *stream);

/* Neighbourhood gather-reduce (the operator Sec. 7 proposes for reductions
 * over neighbour lists): for each vertex v of a set, out[v] = the
 * reduction, over the entries e = (v, u) of v's row (its out-neighbours;
 * its in-neighbours on a symmetric CSR), of
 *   GR_REDUCE_SUM   x[u]            (x, out: double)
 *   GR_REDUCE_WSUM  w(e) * x[u]     (double; needs edge weights)
 *   GR_REDUCE_MIN   x[u]            (x, out: int32)
 *   GR_REDUCE_MAX   x[u]            (int32)
 * A vertex without entries gets the identity: 0, INT32_MAX or INT32_MIN.
 * The set is every vertex (frontier NULL) or the q distinct vertices of
 * frontier[q] (device int32; a repeated vertex makes its sum undefined);
 * out entries of vertices outside the set are left as they are. x[n] must
 * be device memory; out[n] is device or host memory. Sums are in FP64 in an
 * order that differs from a sequential loop (rounding at the level of
 * FP64's epsilon times the row's absolute sum); min and max are exact. */
enum { GR_REDUCE_SUM = 0, GR_REDUCE_WSUM = 1, GR_REDUCE_MIN = 2, GR_REDUCE_MAX = 3 };
gr_status gr_neighbor_reduce(gr_graph *g, int32_t op, const int32_t *frontier, int32_t q,
                             const void *x, void *out, void *stream);

/* Node rankings on a bipartite graph (Sec. 5.5 "Bipartite graphs": the
 * HITS, SALSA and personalized-PageRank rankings of the who-to-follow
 * computation the paper cites, each iteration a 2-hop traversal hub ->
 * authority -> hub). The graph is given as a symmetric CSR whose vertices
 * [0, n_left) are hubs and [n_left, n) authorities, every entry joining a
 * hub and an authority (else GR_EINVAL). score[n] (double, device or host)
 * receives the hub scores on [0, n_left) and the authority scores on
 * [n_left, n).
 *   gr_hits   Kleinberg: a[r] = sum of h[l] over the hubs l linked to r,
 *             then h[l] = sum of a[r] over the authorities r linked to l,
 *             each vector scaled to unit Euclidean length after its update
 *             (left as is if zero); h starts at 1/sqrt(n_left), a at 0.
 *   gr_salsa  Lempel and Moran: a[r] = sum of h[l] / deg(l), then
 *             h[l] = sum of a[r] / deg(r); h starts at 1/(hubs with links)
 *             on those hubs, 0 elsewhere.
 * Both stop after max_iter iterations or once the summed absolute change of
 * all scores in an iteration is below tol; *iters (host, may be NULL;
 * asking for it synchronises) receives the iterations run. FP64, one
 * cooperative kernel for the whole iteration loop. */
gr_status gr_hits(gr_graph *g, int32_t n_left, int32_t max_iter, double tol, double *score,
                  int32_t *iters, void *stream);
gr_status gr_salsa(gr_graph *g, int32_t n_left, int32_t max_iter, double tol, double *score,
                   int32_t *iters, void *stream);

/* Personalized PageRank (the PageRank iteration of gr_pagerank with the
 * teleport and the dangling mass sent uniformly to the seeds instead of all
 * vertices): r'[v] = (1 - damping) t[v] + damping * (sum over entries (v, u)
 * of r[u]/deg(u) + D t[v]), t = 1/num_seeds on each seed, D = the rank mass
 * on degree-0 vertices, r0 = t. seeds[num_seeds] (host, distinct, in
 * [0, n)). The CSR must be symmetric (the gather runs over rows). Stops as
 * gr_hits does; rank[n] (double, device or host); FP64. */
gr_status gr_ppr(gr_graph *g, const int32_t *seeds, int32_t num_seeds, double damping,
                 int32_t max_iter, double tol, double *rank, int32_t *iters, void *stream);

/* BFS that allocates nothing, for callers that cannot call cudaMalloc:
 * code running while a CUDA stream is being captured into a graph (an
 * allocation there breaks the capture), hosts whose device memory is owned
 * by their own allocator or pool, and real-time loops that forbid
 * allocation after start-up. The paper has no counterpart; it runs a
 * push-only cooperative BFS kernel (one launch, a bounded grid barrier per
 * level) and gives the same depths as gr_bfs.
 *
 * row_off[n+1] and col[m] are device pointers to a CSR as described above,
 * read but not validated (a column index outside [0, n) is skipped);
 * depth[n] and parent[n] (parent may be NULL) are device pointers receiving
 * the same results as gr_bfs. A traversal cut short on the device (a grid
 * barrier wait that ran out) leaves depth[src] = GR_NOALLOC_INCOMPLETE
 * instead of 0: check depth[src] after synchronising `stream` where that
 * matters, since the call itself returns before the work runs. n must not exceed
 * 1048576 (1 << 20): the scratch is one fixed device array of about 8.5 MB
 * (control block, two frontier queues, visited bitmap) that every GPU which
 * loads this library holds until the process exits; larger n returns
 * GR_EINVAL. The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) with that device current, and looks it up
 * again after the device's context changed (cudaDeviceReset); make that
 * first call before any stream capture. All calls on a device share the array and
 * each call reinitialises what it reads, so calls that overlap on the GPU
 * (other streams, other threads) race and must be ordered by the caller.
 * Work is enqueued on `stream`; nothing is synchronised. */
#define GR_NOALLOC_INCOMPLETE (-2)
gr_status gr_bfs_noalloc(int32_t n, int64_t m, const int32_t *row_off,
                         const int32_t *col, int32_t src, int32_t *depth,
                         int32_t *parent, void *stream);

/* Per-level trace of the last completed gr_bfs (every level-loop driver;
 * host outputs, any may be NULL; synchronises). For level i < min(cap,
 * *levels): dir[i] 0 = push, 1 = pull; frontier[i] the frontier size the
 * level expanded; edges[i] that frontier's edge count; end_us[i] device
 * time (globaltimer) from the end of initialisation to the end of level i,
 * in microseconds. At most 64 levels are recorded. */
gr_status gr_bfs_trace(gr_graph *g, int32_t cap, int32_t *dir, int32_t *frontier,
                       int64_t *edges, double *end_us, int32_t *levels);

/* Autotuning (the paper leaves these knobs to the user, Sec. 4.4, and notes
 * that the best strategy follows from the degree distribution, Sec. 6). A
 * graph starts with settings derived from its degree statistics;
 * gr_autotune times candidate settings on the k >= 1 sample sources srcs
 * (host array) with CUDA events and keeps the fastest, per graph:
 * GR_TUNE_BFS tunes the level-loop driver, the persistent grid size and the
 * push/pull thresholds; GR_TUNE_SSSP the near/far bucket width. Options
 * passed as 0 use the tuned values. Results never depend on tuning.
 * Synchronises. */
enum { GR_TUNE_BFS = 1, GR_TUNE_SSSP = 2 };
gr_status gr_autotune(gr_graph *g, const int32_t *srcs, int32_t k, int32_t what,
                      void *stream);

/* The graph's current tuned settings (host outputs; times may be NULL and
 * are 0 until measured): mode, alpha, beta, block (blocks per SM of the
 * persistent kernel, 0 = all resident) and delta; mean time per BFS / SSSP
 * over the tuning sample. */
gr_status gr_tuned_opts(const gr_graph *g, gr_opts *out, double *bfs_ms, double *sssp_ms);

/* The graph's current SSSP settings (host outputs, any may be NULL): the
 * level-loop driver (GR_MODE_*), blocks per SM of the persistent kernel
 * (0 = all resident) and the near/far bucket width (UINT32_MAX: one bucket). */
gr_status gr_tuned_sssp(const gr_graph *g, int32_t *mode, int32_t *blocks_per_sm,
                        uint32_t *delta);

/* ------------------------------------------------------------------------
 * Query server (not in the paper): BFS / SSSP / CC queries on resident
 * graphs with continuous batching. One worker slot owns a CUDA stream and
 * per-graph workspaces and runs one batch at a time. Admission: a batch is
 * started when its result buffers (4n bytes per request) and any workspace
 * it must create fit in the device-memory budget next to the workspaces
 * the slot already keeps (workspaces stay until the server is destroyed);
 * requests are taken in arrival order, and the oldest one starts alone
 * even when it does not fit while nothing is in flight, so the budget
 * bounds batching, not single requests. A BFS request on a batchable graph
 * takes up to max_batch - 1 further queued BFS requests for that graph and
 * runs them as lanes of one gr_bfs_batch traversal (see
 * gr_server_add_graph for when); likewise an SSSP request takes further
 * queued SSSP requests for its graph as lanes of one gr_sssp_batch search
 * (up to max_batch and the graph's lane limit, which keeps that search's
 * scratch within 4 GiB). The queued CC requests of a graph (whose answers
 * are all the same) share one gr_cc run and one result buffer, up to
 * max_batch of them. Results equal those of gr_bfs / gr_sssp / gr_cc
 * alone. Traversals use each graph's tuned driver. With max_batch = 1 the
 * server is the plain path: one query per launch sequence, in arrival
 * order, on one stream. A request whose traversal stops at a device-side
 * level or iteration limit fails with GR_ETIMEOUT. Whatever a batch's
 * outcome, the slot waits for the device work it enqueued before it
 * reuses or frees any buffer; it waits at most 120 s, after which that
 * batch fails with GR_ETIMEOUT and the slot fails its later requests
 * (its stream may still hold work, so its buffers are then left alone).
 * The server takes each graph's lock while it enqueues work on the graph.
 * ---------------------------------------------------------------------- */
typedef struct gr_server gr_server;

enum { GR_QUERY_BFS = 0, GR_QUERY_SSSP = 1, GR_QUERY_CC = 2 };

/* budget_bytes > 0; num_slots must be 1 (several slots running traversals
 * at once are disabled: a device fault seen with them is not explained);
 * max_batch in [1, 64]. */
gr_status gr_server_create(size_t budget_bytes, int32_t num_slots, int32_t max_batch,
                           gr_server **out);

/* Register a graph (it must outlive the server) before the first submit.
 * batchable in [0, 64]: 0 keeps the graph's BFS and SSSP requests single;
 * otherwise SSSP requests batch whatever is queued, and a BFS request on
 * the graph runs as a lane of a batch when at least `batchable` BFS
 * requests for the graph (itself included) are queued. 1 batches whatever
 * is queued
 * (low-diameter graphs); a larger value suits graphs with many levels,
 * whose batched traversal costs a host round trip per level and pays only
 * when it carries enough queries. */
gr_status gr_server_add_graph(gr_server *s, gr_graph *g, int32_t batchable,
                              int32_t *graph_id);

/* Queue a query: kind GR_QUERY_BFS (depth), GR_QUERY_SSSP (dist, uint32)
 * or GR_QUERY_CC (labels; src ignored). out (n int32/uint32, device or host
 * memory, may be NULL to discard) receives the result before the request
 * counts as done. *ticket identifies the request. Never blocks. */
gr_status gr_server_submit(gr_server *s, int32_t graph_id, int32_t kind, int32_t src,
                           void *out, uint64_t *ticket);

/* Wait for one request (timeout_ms < 0: no limit; GR_ETIMEOUT on expiry)
 * and forget it; *latency_ms (may be NULL) = submission to completion. */
gr_status gr_server_wait(gr_server *s, uint64_t ticket, int32_t timeout_ms,
                         double *latency_ms);

/* Wait until every submitted request has finished (GR_ETIMEOUT on expiry). */
gr_status gr_server_drain(gr_server *s, int32_t timeout_ms);

/* Totals since creation (host scalars, any may be NULL): completed and
 * failed requests, device launches (a batch counts once), throughput from
 * the first submission to the last completion, latency percentiles (ms,
 * submission to completion) and the mean number of requests per launch. */
gr_status gr_server_stats(gr_server *s, int64_t *completed, int64_t *failed,
                          int64_t *launches, double *qps, double *p50_ms, double *p99_ms,
                          double *mean_batch);

/* Stop the workers (queued requests are dropped) and free the server. */
gr_status gr_server_destroy(gr_server *s);

/* Diagnostics for failure handling (no GPU fault is ever provoked).
 * gr_diag_wait_timeout: a kernel spins on a flag that nothing sets, with
 * the library's bounded-wait logic and a limit of spin_limit polls (in
 * [0, 2^24]); returns GR_ETIMEOUT when the wait gave up, as every bounded
 * device wait of the library reports it, and the context stays usable.
 * gr_diag_fail_alloc: after `after` more successful device allocations the
 * library's allocations fail with GR_ENOMEM (after < 0 restores normal
 * behaviour); process-wide. */
gr_status gr_diag_wait_timeout(int64_t spin_limit, void *stream);
gr_status gr_diag_fail_alloc(int64_t after);

/* Bounds-guard report of a library built with GR_CHECKED (a diagnostic
 * build whose kernels check every data-dependent index, record the first
 * one outside its buffer and skip that access): *site identifies the
 * access (0: no violation), *index and *bound the offending index and its
 * buffer length. Normal builds always report 0. */
gr_status gr_diag_guard(int32_t *site, int64_t *index, int64_t *bound);

/* This thread's last error message ("" if none). The pointer stays valid
 * until this thread's next gr_* call. */
const char *gr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GR_H */
