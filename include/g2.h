/*
 * g2.h — C ABI of libg2.so: frontier-driven edge traversal on one GB300 GPU.
 *
 * The operator at the centre is edgeset.apply / applyModified of the paper's
 * algorithm language (Sec. IV, Fig. 2): for every arc u->v whose source u is
 * in the input vertexset (".from(frontier)") and whose destination passes the
 * destination filter (".to(filter)"), apply an update function to v; with
 * applyModified, return the vertexset of destinations whose tracked value
 * changed.  How it runs on the GPU is chosen by a schedule mirroring the
 * paper's GPU scheduling language (Sec. V, Tables II and III).  BFS, CC,
 * delta-stepping SSSP, PageRank and betweenness centrality (Sec. VII) are
 * built on it.
 *
 * Conventions for every call:
 *  - Pointers named "device" must point to memory of the current CUDA device
 *    (e.g. torch tensors); "host" pointers to ordinary host memory.  Output
 *    arrays are owned by the caller and must hold the stated length.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is issued on that stream; every call returns only after its work has
 *    completed (the host needs frontier sizes, and device-side time-outs are
 *    reported as a status).
 *  - Argument errors return G2_EINVAL before any launch and leave outputs
 *    untouched.  After a device-side failure (G2_ETIMEOUT, G2_EOVERFLOW,
 *    G2_ECUDA) output contents are unspecified.  g2_last_error() returns a
 *    thread-local message for the last failing call on the calling thread.
 *  - Vertex ids are int32 in [0, n); arc counts must be < 2^31.
 *  - One g2_graph handle must not be used by two calls at the same time (its
 *    workspace is shared by the calls made on it); g2_graph_view() gives
 *    another handle on the same topology with a workspace of its own.
 */
#ifndef G2_H
#define G2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
typedef enum {
    G2_OK = 0,
    G2_EINVAL = 1,        /* bad argument (null pointer, id out of range, bad schedule) */
    G2_ENOMEM = 2,        /* device or host allocation failed */
    G2_ECUDA = 3,         /* a CUDA runtime call or kernel failed */
    G2_ETIMEOUT = 4,      /* a bounded device-side wait (grid barrier) ran out */
    G2_EUNSUPPORTED = 5,  /* the schedule combination is not implemented */
    G2_EOVERFLOW = 6      /* a queue or a value exceeded its capacity / range */
} g2_status;

/* ---------------------------------------------------------- load flags */
#define G2_SYMMETRIC   0x1u  /* every arc u->v has v->u (then CSC aliases CSR) */
#define G2_DEVICE_PTRS 0x2u  /* rowptr/col/w are device pointers (else host) */
#define G2_PREPARE_PAGERANK 0x4u /* build PageRank's layouts in the background */
#define G2_LOAD_OVERLAP 0x8u     /* the load runs beside other GPU work: pinned or device
                                    arrays go by copy engine, leaving the SMs */

/* --------------------------------------------- schedule (Table II fields) */
/* configLoadBalance load_balance_type */
#define G2_LB_VERTEX_BASED 0 /* default: one thread per active vertex */
#define G2_LB_CM 1           /* CTA mapping: a CTA takes a chunk of vertices, balances its edges */
#define G2_LB_WM 2           /* warp mapping: a warp takes a chunk of vertices, balances its edges */
#define G2_LB_STRICT 3       /* equal arc count per thread over a frontier-wide prefix sum */
#define G2_LB_EDGE_ONLY 4    /* edge-parallel over all arcs (COO); needs the all-vertices frontier */
#define G2_LB_ETWC 5         /* ETWC, Algorithm 3: thread/warp/CTA split inside each CTA */
#define G2_LB_TWC 6          /* TWC: frontier-wide degree buckets for thread, warp, CTA */
/* configDirection */
#define G2_PUSH 0
#define G2_PULL 1
/* configDirection front_rep (input frontier representation when PULL) */
#define G2_BOOLMAP 0
#define G2_BITMAP 1
/* configFrontierCreation */
#define G2_FUSED 0
#define G2_UNFUSED_BOOLMAP 1
#define G2_UNFUSED_BITMAP 2
/* configDeduplication */
#define G2_DEDUP_ENABLED 0
#define G2_DEDUP_DISABLED 1
#define G2_DEDUP_MONOTONIC_COUNTERS 0
#define G2_DEDUP_BITMAP 1
#define G2_DEDUP_BOOLMAP 2

/* SimpleGPUSchedule (Sec. V, Table II).  An all-zero struct is the paper's
 * default schedule: VERTEX_BASED, no blocking, PUSH, BOOLMAP pull input,
 * FUSED frontier creation, deduplication ENABLED with MONOTONIC_COUNTERS,
 * delta 1, kernel fusion DISABLED. */
typedef struct {
    int32_t load_balance;      /* G2_LB_* */
    int32_t edge_blocking;     /* 1 = EdgeBlocking (Algorithms 1-2); EDGE_ONLY full sweeps only */
    int32_t blocking_size;     /* vertices per EdgeBlocking segment; 0 = derived from L2 size */
    int32_t direction;         /* G2_PUSH / G2_PULL */
    int32_t pull_frontier;     /* G2_BOOLMAP / G2_BITMAP: input representation for PULL */
    int32_t frontier_creation; /* G2_FUSED / G2_UNFUSED_BOOLMAP / G2_UNFUSED_BITMAP */
    int32_t dedup;             /* G2_DEDUP_ENABLED / G2_DEDUP_DISABLED */
    int32_t dedup_type;        /* G2_DEDUP_MONOTONIC_COUNTERS / _BITMAP / _BOOLMAP */
    int32_t delta;             /* configDelta: priority bucket width (0 = 1) */
    int32_t kernel_fusion;     /* configKernelFusion: 1 = whole loop in one persistent kernel */
} g2_schedule;

/* HybridGPUSchedule (Sec. V, Table III).  criteria G2_CRITERIA_NONE: always
 * s1.  G2_INPUT_VERTEXSET_SIZE: s1 when |input frontier| < threshold * n,
 * else s2 (threshold read as a fraction of the vertex count).  With kernel
 * fusion (s1.kernel_fusion) the whole loop is one persistent kernel that runs
 * s1's rounds throughout: the criterion is not evaluated inside it, and for
 * a hybrid criterion s2 must request fusion too (G2_EUNSUPPORTED otherwise). */
#define G2_CRITERIA_NONE 0
#define G2_INPUT_VERTEXSET_SIZE 1
typedef struct {
    int32_t criteria;
    float threshold;
    g2_schedule s1, s2;
} g2_hybrid;

/* ---------------------------------------------------------------- graph */
typedef struct g2_graph g2_graph;

/* g2_load_csr — copy a CSR graph to the device (Sec. VI-C: the host side
 * loads the graph and allocates the data structures).
 *   n        vertex count, 0 <= n < 2^31-1
 *   m        arc count, 0 <= m < 2^31
 *   rowptr   int32[n+1], rowptr[0] = 0, non-decreasing, rowptr[n] = m
 *   col      int32[m] arc heads; each list sorted ascending, no duplicates
 *   w        int32[m] arc weights (>= 1 for SSSP) or NULL
 *   flags    G2_SYMMETRIC | G2_DEVICE_PTRS | G2_PREPARE_PAGERANK | G2_LOAD_OVERLAP
 *   stream   stream for the copies and validation
 *   out      receives the handle (library-owned; free with g2_free_graph)
 * The input arrays are copied; the caller may free them after return.  The
 * layout is validated on the device (G2_EINVAL if rowptr is not monotone,
 * an id is out of range, a list is unsorted / has duplicates or a weight is
 * negative).  Where the device can read the caller's arrays directly (device
 * memory, pinned host memory, or pageable host memory on a system whose GPU
 * reads it through the host page tables, as over the Grace-Blackwell
 * coherent link) and col / w are 16-byte aligned, one kernel reads, checks
 * and stores the arcs; otherwise they are copied with cudaMemcpyAsync and
 * checked after.  G2_LOAD_OVERLAP (a load on its own stream while other
 * calls run, e.g. the next graph of a stream of requests) copies pinned host
 * or device arrays with a copy engine and validates them in one pass after,
 * so the other calls keep every SM during the transfer (a kernel that needs
 * whole SMs would otherwise wait for the copy kernel's); pageable arrays in
 * such a load are read by the copy kernel on a quarter of the SMs.  For a
 * non-symmetric graph the transpose (CSC, lists sorted
 * ascending) is built on the host for the PULL direction.  Device memory
 * comes from the library's stream-ordered pool (see g2_free_graph).
 * G2_PREPARE_PAGERANK: the layouts the tuned PageRank sweep needs (the
 * source-blocked arcs and the rank order of the vertices) are built
 * after the load returns, by a host thread on a stream of its own (with the
 * priority of the load's stream), while the caller's next calls run;
 * g2_pagerank (and g2_free_graph) wait for them.
 * Without the flag the first g2_pagerank builds them. */
g2_status g2_load_csr(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *col,
                      const int32_t *w, uint32_t flags, void *stream, g2_graph **out);
/* g2_free_graph — release a handle (a graph or a view); the topology goes
 * when its last handle does (the host side of the generated code frees the
 * graph's device arrays, Sec. VI-C).  No call on the handle may be in progress.  The
 * device memory returns to the library's per-device stream-ordered pool,
 * which keeps it for later loads instead of handing it back to the driver
 * (no cudaFree, no device-wide synchronisation).  NULL is ignored. */
void g2_free_graph(g2_graph *g);

/* g2_graph_view — a second handle on g's device topology with a workspace of
 * its own, so that two streams can run queries on one graph concurrently.
 * The topology is reference-counted; free each view with g2_free_graph. */
g2_status g2_graph_view(g2_graph *g, g2_graph **out);

/* g2_graph_info — vertex and arc counts, device id, SM count and L2 bytes. */
g2_status g2_graph_info(const g2_graph *g, int64_t *n, int64_t *m, int32_t *sm_count,
                        int64_t *l2_bytes);

/* g2_edge_block — EdgeBlocking preprocessing, Algorithm 1 (Sec. VI-D), on the
 * device: the arcs regrouped into segments of N destination vertices
 * (segment floor(dst/N)), input (CSR) order kept inside a segment.  Stored in
 * the handle for later EDGE_ONLY + blocking sweeps; a different N rebuilds.
 * N <= 0 derives N from the L2 size.  *num_segments receives the segment
 * count (nullable). */
g2_status g2_edge_block(g2_graph *g, int32_t N, int32_t *num_segments, void *stream);

/* g2_edge_block_export — copy the blocked COO built by g2_edge_block into
 * caller device buffers: src[m], dst[m] int32 and seg_end[num_segments+1]
 * int64 (seg_end[s] = one past the last arc of segment s; last entry = m). */
g2_status g2_edge_block_export(g2_graph *g, int32_t *src, int32_t *dst, int64_t *seg_end,
                               void *stream);

/* ------------------------------------------------------------- frontiers */
#define G2_FRONTIER_SPARSE 0  /* SparseQueue: int32 vertex list */
#define G2_FRONTIER_BITMAP 1  /* one bit per vertex */
#define G2_FRONTIER_BOOLMAP 2 /* one byte per vertex */
typedef struct g2_frontier g2_frontier;

/* A vertexset of graph g in the given representation, initially empty.
 * Library-owned and reusable across calls (the frontier reuse of Sec. VI-A). */
g2_status g2_frontier_create(g2_graph *g, int32_t format, g2_frontier **out);
void g2_frontier_free(g2_frontier *f);
/* Replace the contents with verts[0..k) (host int32, duplicates allowed only
 * for SPARSE, where they are kept). */
g2_status g2_frontier_set(g2_frontier *f, const int32_t *verts, int32_t k, void *stream);
/* Number of vertices in f (for SPARSE: the list length). */
g2_status g2_frontier_size(g2_frontier *f, int32_t *size, void *stream);
/* Write the members of f into verts (device int32, capacity cap) in
 * unspecified order; *k receives the count (G2_EOVERFLOW if > cap). */
g2_status g2_frontier_list(g2_frontier *f, int32_t *verts, int32_t cap, int32_t *k, void *stream);

/* ------------------------------------------------------ edgeset.apply */
/* Update functions (the UDFs of Sec. IV with the atomics of Sec. VI-B):
 *  G2_OP_BFS        vdata int32 depth[n] (-1 = unvisited), vdata2 int32
 *                   parent[n] or NULL.  Filter: depth[v] == -1.  Update:
 *                   depth[v] = depth[u] + 1 (compare-and-swap in PUSH),
 *                   parent[v] = smallest such u.  Output: v newly visited.
 *  G2_OP_RELAX_MIN  vdata int32 dist[n] (INT32_MAX = unreached); needs arc
 *                   weights.  dist[v] = min(dist[v], dist[u] + w(u,v)).
 *                   Output: v whose dist decreased.
 *  G2_OP_LABEL_MIN  vdata int32 label[n].  label[v] = min(label[v], label[u]).
 *                   Output: v whose label decreased.
 *  G2_OP_PR_ADD     vdata float contrib[n] (per source), vdata2 float acc[n].
 *                   acc[v] += contrib[u].  No output frontier (out must be NULL).
 *  G2_OP_BC_SIGMA   vdata int32 depth[n] (read only), vdata2 double sigma[n].
 *                   If depth[v] == depth[u] + 1: sigma[v] += sigma[u].  No output.
 *                   (The forward path counts of Brandes' BC, Sec. VII.)
 *  G2_OP_BC_DELTA   Brandes' dependency step of one level (Sec. VII, BC):
 *                   the input vertexset is level d + 1 of a BFS; vdata int32
 *                   depth[n] (read only), vdata2 double[2n] = sigma[0..n)
 *                   (read only) followed by delta[n..2n) (accumulated).  Over
 *                   an arc w->v with w in the input and depth[v] == depth[w] - 1:
 *                   delta[v] += sigma[v] / sigma[w] * (1 + delta[w]).  Needs
 *                   a symmetric graph (the arcs out of level d + 1 are the
 *                   reverses of the shortest-path arcs into it; G2_EINVAL
 *                   else).  No output.  Run from the deepest level up, it
 *                   leaves delta_s(v) for every v != s. */
typedef enum {
    G2_OP_BFS = 0,
    G2_OP_RELAX_MIN = 1,
    G2_OP_LABEL_MIN = 2,
    G2_OP_PR_ADD = 3,
    G2_OP_BC_SIGMA = 4,
    G2_OP_BC_DELTA = 5
} g2_op;

/* g2_edgeset_apply — one edgeset.from(in).to(filter).apply[Modified](op).
 *   in        input vertexset, or NULL for all vertices
 *   vdata/2   device arrays, typed by op (above)
 *   sched     schedule (NULL = defaults); a hybrid picks s1/s2 by |in|
 *   out       output vertexset (applyModified), or NULL (apply).  Its
 *             previous contents are replaced.
 *   out_size  host int32 receiving |out| (nullable) */
g2_status g2_edgeset_apply(g2_graph *g, g2_op op, g2_frontier *in, void *vdata, void *vdata2,
                           const g2_hybrid *sched, g2_frontier *out, int32_t *out_size,
                           void *stream);

/* -------------------------------------------------------------- algorithms */
/* Schedules: a non-NULL `sched` runs exactly that schedule (a simple one, or a
 * hybrid choosing s1/s2 each round by the input vertexset size).  NULL selects
 * the library's tuned schedule for the algorithm, stated with each call. */
/* BFS (Fig. 2): depth int32[n] device (-1 unreachable), parent int32[n]
 * device or NULL (parent[src] = src, else the smallest-id in-neighbour one
 * level up, -1 unreachable).  Loop until the frontier is empty.  With kernel
 * fusion the whole loop is one persistent cooperative kernel; fused WM runs
 * the levels of up to 1024 vertices per cluster CTA (16384 with 16-CTA
 * clusters) inside one thread-block cluster and hands larger levels to the
 * grid-wide kernel (back below half that size), one launch per hand-over.
 * A hybrid with kernel fusion on both schedules and s2 VERTEX_BASED PULL over
 * a bitmap runs in one cooperative kernel too, choosing the direction per
 * level; its PUSH half is VERTEX_BASED, WM, CM, ETWC (CTA-stage entries of
 * 4096 arcs or more go to a grid-wide pass inside the launch) or STRICT (the
 * prefix sum of the level's degrees taken over the grid inside the launch).
 * NULL schedule: that fused direction-optimising hybrid, STRICT PUSH below 2%
 * of n, VERTEX_BASED PULL over a bitmap otherwise; on a bounded-degree graph
 * (largest out-degree <= 32: road networks, meshes) fused WM PUSH instead. */
g2_status g2_bfs(g2_graph *g, int32_t src, int32_t *depth, int32_t *parent,
                 const g2_hybrid *sched, void *stream);

/* Connected components (Soman et al., Sec. VII): label int32[n] device,
 * label[v] = smallest vertex id in v's component (arcs taken as undirected).
 * With a schedule: rounds of hooking along the arcs of the active vertices
 * (PUSH, an edgeset.apply with the schedule's load balancing) or min-label
 * propagation (PULL), each followed by pointer jumping to the roots; active =
 * vertices whose label changed.  NULL schedule: lock-free linking with
 * neighbour sampling (two sampled arcs per vertex, then the remaining arcs of
 * the vertices outside the largest component), then pointer jumping.  Needs a
 * symmetric graph (G2_EINVAL else). */
g2_status g2_cc(g2_graph *g, int32_t *label, const g2_hybrid *sched, void *stream);

/* Delta-stepping SSSP with a two-bucket (near/far) priority queue
 * (Sec. III and V, configDelta): dist int32[n] device, INT32_MAX unreachable.
 * delta > 0 overrides the schedule's delta.  Needs weights >= 1.
 * G2_EOVERFLOW if a distance would reach INT32_MAX.  With kernel fusion and
 * WM, buckets run inside one thread-block cluster (near lists and far piles in
 * shared memory) while near rounds hold at most 1,024 vertices per cluster CTA,
 * and in the grid-wide kernel otherwise (back at a bucket boundary with a
 * small far pile), one launch per hand-over.  NULL schedule: STRICT PUSH,
 * unfused; fused WM PUSH on a bounded-degree graph (largest out-degree <= 32). */
g2_status g2_sssp_delta(g2_graph *g, int32_t src, int32_t delta, int32_t *dist,
                        const g2_hybrid *sched, void *stream);

/* PageRank, topology-driven (Sec. VII): rank float[n] device.  x0 = 1/n;
 * each round x'[v] = (1-d)/n + d*(sum_{u->v} x[u]/outdeg(u) + D/n), D = the
 * total rank of vertices without out-arcs.  `iters` rounds, no convergence
 * test.  PULL + EDGE_ONLY (and NULL): the source-blocked sweep (EdgeBlocking,
 * Sec. VI-D, applied to the pull's sources: blocks of 49,152 sources ranked by
 * degree, whose shares one CTA holds in shared memory, one reduction per run
 * of a destination's arcs within a block; the layout is built on the first
 * call, or in the background with G2_PREPARE_PAGERANK), or where that layout
 * does not apply (more than 1,024 blocks) arc-balanced segmented sums over
 * the CSC; PULL + VERTEX_BASED/WM/CM: per-destination sums; PUSH (any load
 * balancing, EDGE_ONLY optionally with EdgeBlocking): arc-parallel atomic
 * adds. */
g2_status g2_pagerank(g2_graph *g, float damping, int32_t iters, float *rank,
                      const g2_hybrid *sched, void *stream);

/* Betweenness centrality (Brandes; Sec. VII and the BC rows of Tables V-VI)
 * summed over the k sources srcs (host int32[k]): bc double[n] device, no
 * normalisation, no halving; per source a forward pass of path counts
 * (G2_OP_BC_SIGMA's update) and a backward pass of dependencies (G2_OP_BC_DELTA's).  Path counts
 * are extended-range numbers (64-bit integer mantissa, int32 exponent per
 * vertex), so
 * they neither overflow nor underflow on high-diameter graphs.  Each level's
 * discovery follows the (hybrid) schedule; with kernel fusion each source
 * runs in one persistent cooperative kernel, and with fused WM on a symmetric
 * bounded-degree graph the levels of at most 256 vertices per cluster CTA run
 * inside one thread-block cluster (forward and backward), the larger ones in
 * the grid-wide kernel.  NULL schedule: the
 * direction-optimising hybrid as per-level launches (STRICT PUSH below 2% of
 * n, VERTEX_BASED PULL); fused WM PUSH on a bounded-degree graph (largest
 * out-degree <= 32). */
g2_status g2_bc(g2_graph *g, const int32_t *srcs, int32_t k, double *bc,
                const g2_hybrid *sched, void *stream);

/* Multi-source BFS (not in the paper: a workload addition, the batched
 * queries of the serving path): k <= 64 sources (host int32[k]) in one traversal, one bit
 * per source in per-vertex 64-bit visit/frontier masks.  depth int32[k][n]
 * device (row i = BFS from srcs[i]).  Schedules: PUSH with any frontier load
 * balancing but EDGE_ONLY, PULL with VERTEX_BASED or WM, or kernel fusion with
 * WM PUSH (the whole loop in one cooperative kernel).  NULL schedule: the
 * direction-optimising hybrid (STRICT PUSH below 2% of n, VERTEX_BASED PULL);
 * on a bounded-degree graph (largest out-degree <= 32) the sources run as
 * single-source fused WM queries, about one per 12 SMs at a time, each on an
 * internal view of the graph and a stream of its own driven by a library
 * thread (their one-cluster loops share the GPU; the caller's stream is
 * synchronised first; G2_BATCH_SPLIT_WORKERS sets the count, 0 runs the
 * fused multi-source loop instead). */
g2_status g2_bfs_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t *depth,
                       const g2_hybrid *sched, void *stream);

/* Multi-source SSSP (not in the paper: a workload addition, the batched
 * queries of the serving path; the queue is Sec. III's delta-stepping):
 * k <= 32 sources, stacked distance arrays dist
 * int32[k][n] device, relaxed together in one frontier loop with the
 * near/far queue of g2_sssp_delta (one bit per source in per-vertex masks).
 * Schedules: PUSH with any frontier load balancing but EDGE_ONLY, or kernel
 * fusion with WM PUSH (the whole loop in one cooperative kernel).  NULL
 * schedule: STRICT PUSH; on a bounded-degree graph (largest out-degree <= 32)
 * the sources run as single-source fused WM queries, about one per 19 SMs at
 * a time, as g2_bfs_batch does (G2_BATCH_SPLIT_WORKERS = 0: the fused
 * multi-source loop). */
g2_status g2_sssp_batch(g2_graph *g, const int32_t *srcs, int32_t k, int32_t delta,
                        int32_t *dist, const g2_hybrid *sched, void *stream);

/* Asynchronous SSSP and BFS (not the paper's method: Sec. VII-A and Table VII
 * show its delta-stepping losing to a 24-core CPU on road graphs, where every
 * bucket and every near round inside it ends at a barrier while the frontier
 * holds a few thousand vertices).  One persistent cooperative kernel relaxes
 * the out-arcs of the vertices in a shared worklist (a vertex queued at most
 * once at a time) with no barrier inside a bucket of width `delta`: a bucket
 * ends when a device-side count of pending items reaches zero, and only the
 * step to the next bucket (the smallest far distance, the split of the far
 * pile) synchronises the grid.  delta <= 0: one bucket, fully asynchronous.
 * Every wait is bounded (G2_ETIMEOUT).  If the worklist (4 n appends) runs
 * out the kernel is run again with four times the room.  Results equal
 * g2_sssp_delta's / g2_bfs's:
 *   g2_sssp_async  dist int32[n] device (INT32_MAX unreachable); needs
 *                  weights >= 1; G2_EOVERFLOW if a distance would reach
 *                  INT32_MAX.
 *   g2_bfs_async   depth int32[n] device (-1 unreachable), parent int32[n]
 *                  device or NULL (the smallest-id in-neighbour one level up,
 *                  taken by a pull pass over the final depths); delta counts
 *                  levels per bucket.
 * g2_last_stats: `iterations` = worklist items processed, `barriers` = grid
 * barriers (three per bucket). */
g2_status g2_sssp_async(g2_graph *g, int32_t src, int32_t delta, int32_t *dist, void *stream);
g2_status g2_bfs_async(g2_graph *g, int32_t src, int32_t delta, int32_t *depth, int32_t *parent,
                       void *stream);

/* g2_bfs_csr_static — BFS that allocates no device memory (the paper has no
 * counterpart: this entry point exists for callers that cannot allocate).
 * For callers that cannot call cudaMalloc, e.g. code running inside another
 * runtime that has reserved the device memory for its own pool, or latency-
 * bound code that cannot afford the device synchronisation allocation may
 * cause.  The caller passes everything in its own memory:
 *   n, m            vertex count (1 <= n <= 1048576) and arc count (< 2^31)
 *   rowptr, col     the graph as a device CSR (int32[n+1], int32[m]); it is
 *                   read, never copied; a check kernel reads it first and
 *                   returns G2_EINVAL, traversing nothing, if a row offset
 *                   is outside [0, m] or decreasing, rowptr[0] != 0,
 *                   rowptr[n] != m, or a column id is outside [0, n)
 *   src             source vertex
 *   depth           int32[n] device output, as g2_bfs
 *   parent          int32[n] device output or NULL, as g2_bfs
 * Scratch (two frontier queues, counters, grid-barrier and error words) is a
 * fixed array of 8 MiB inside the library that every GPU which loads the
 * library holds until the process exits; n above its capacity returns
 * G2_EINVAL.  The first call on a device resolves that array's device address
 * (make that first call before any stream capture); under CUDA's lazy module
 * loading that first call also loads the module holding the array, which
 * reserves its device memory and may synchronise the device, so a caller that
 * cannot afford that makes one call at set-up time.  All calls share the one
 * array, so calls that overlap on the GPU (two streams, or two threads) race
 * and must be serialised by the caller.  The call reads 64 bytes of status
 * back into host stack memory (a pageable copy, which can wait behind other
 * copies in flight on the device) and returns after completion. */
g2_status g2_bfs_csr_static(int32_t n, int64_t m, const int32_t *rowptr, const int32_t *col,
                            int32_t src, int32_t *depth, int32_t *parent, void *stream);

/* ----------------------------------------------------------- diagnostics */
/* Counters of the last algorithm call made on this thread. */
typedef struct {
    int32_t iterations;     /* frontier rounds (or PR rounds, CC rounds, buckets) */
    int32_t push_rounds;    /* rounds run PUSH */
    int32_t pull_rounds;    /* rounds run PULL */
    int32_t launches;       /* kernels launched (not counting the one-warp kernels that
                               store a call's few host-side values, e.g. the source) */
    int64_t arcs_examined;  /* arcs read by the traversal (0 unless counted) */
    int32_t barriers;       /* grid or cluster barriers passed in fused kernels */
    int32_t reserved;
} g2_stats;
g2_status g2_last_stats(g2_stats *out);
/* Count arcs examined in later calls on this thread (costs one atomic per
 * CTA per launch). */
void g2_set_count_arcs(int32_t enable);

/* Kernel timing (diagnostic, off by default): when enabled, CUDA events are
 * recorded on the call's stream around every launch of the named hot kernels
 * ("pr_round" PageRank arc sweep, "pr_vertex" its vertex pass, "bfs_push",
 * "bfs_pull", "cc_hook", "sssp_relax")
 * and their durations accumulated per name on the calling thread.
 * g2_kernel_time returns the total milliseconds and launch count for `name`
 * since the last reset; reset != 0 clears every name afterwards. */
void g2_set_kernel_timing(int32_t enable);
g2_status g2_kernel_time(const char *name, double *ms, int64_t *launches, int32_t reset);

const char *g2_last_error(void);

/* Self-test of the bounded device-side wait used by grid barriers: a kernel
 * waits on a flag that nothing sets, for at most limit_ns nanoseconds, then
 * records a time-out and returns.  Returns G2_ETIMEOUT when that works. */
g2_status g2_selftest_wait_timeout(int64_t limit_ns, void *stream);

/* Library version string. */
const char *g2_version(void);

#ifdef __cplusplus
}
#endif
#endif /* G2_H */
