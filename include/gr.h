/*
 * gr.h — C ABI of the GB300 frontier-traversal library.
 *
 * The library implements the data-parallel hot path of the frontier
 * abstraction of Wang et al., "Gunrock: GPU Graph Analytics" (ACM TOPC 2017):
 * the advance operator (Sec. 4.1, Sec. 5.1), the filter operator (Sec. 4.2,
 * Sec. 5.2.1), and the two primitives they drive, breadth-first search with
 * the direction-optimising pull step (Sec. 6.1, Sec. 5.1.4, Alg. 2) and
 * single-source shortest paths with integer weights and a near/far priority
 * queue (Sec. 3 example, Alg. 1, Sec. 5.1.5, Sec. 6.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Graphs are CSR with int32 row offsets R (n+1 entries, R[0] = 0,
 *    R[n] = m, non-decreasing) and int32 column indices C (m entries, each in
 *    [0, n)), optionally uint32 weights W (m entries, each >= 1).
 *  - Every pointer to per-vertex or per-edge data is a DEVICE pointer owned by
 *    the caller unless stated otherwise; the library never frees it.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Entry points are asynchronous on that stream unless marked
 *    "synchronous".
 *  - Results: unreachable vertices get depth -1, dist GR_INF_DIST (UINT32_MAX)
 *    and pred -1; the source gets depth 0, dist 0, pred -1 (Alg. 1
 *    Set_Problem_Data).
 *  - Argument errors are returned synchronously.  Errors the GPU detects
 *    while running (capacity exceeded, distance overflow, barrier timeout)
 *    are recorded in a device status word of the workspace and reported by
 *    gr_sync_status().  The library never traps or asserts on the device.
 *  - Thread safety: a gr_graph is immutable after creation and may be shared
 *    by concurrent calls (gr_bfs_multi, whose scratch is per graph, takes a
 *    per-graph lock); a gr_workspace must be used by one call at a time
 *    (calls on different streams need different workspaces).
 */
#ifndef GR_H_
#define GR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef int32_t gr_status;
#define GR_OK                 0
#define GR_ERR_INVALID_ARG   -1  /* bad pointer, size, source or mode        */
#define GR_ERR_OOM           -2  /* device allocation failed                  */
#define GR_ERR_CUDA          -3  /* a CUDA runtime call failed                */
#define GR_ERR_CAPACITY      -4  /* an output buffer was too small            */
#define GR_ERR_OVERFLOW      -5  /* a distance does not fit below UINT32_MAX  */
#define GR_ERR_TIMEOUT       -6  /* a device-side wait ran out of iterations  */
#define GR_ERR_INVALID_GRAPH -7  /* CSR failed validation                     */
#define GR_ERR_UNSUPPORTED   -8  /* mode not available for this graph         */

#define GR_INF_DIST 0xFFFFFFFFu

/* Human-readable name of a status code (static string, never NULL). */
const char* gr_status_str(gr_status s);

/* Library ABI version: (major << 16) | minor. */
int32_t gr_version(void);

/* ---- graph ------------------------------------------------------------- */
typedef struct gr_graph gr_graph;
typedef struct gr_workspace gr_workspace;

/* gr_graph_create_csr flags */
#define GR_BORROW    0u  /* keep the caller's device arrays (caller keeps them alive) */
#define GR_COPY      1u  /* copy R, C, W into device memory the graph owns            */
#define GR_SYMMETRIC 2u  /* caller asserts (u,v) in E => (v,u) in E with equal weight;
                            verified on the device; enables the pull step         */

/*
 * Create a graph handle over a device CSR (Sec. 5.4: CSR row offsets R and
 * column indices C; per-edge data as a structure of arrays).
 *   n >= 0 vertices, m >= 0 directed entries, n and m below 2^31.
 *   row_offsets: device int32[n+1]; cols: device int32[m];
 *   weights: device uint32[m] or NULL (needed only by SSSP).
 * Validates on the device and is synchronous on `stream`: returns
 * GR_ERR_INVALID_GRAPH if R[0] != 0, R[n] != m, R decreases, a column is
 * outside [0, n), a weight is 0, or (with GR_SYMMETRIC) some row is not
 * strictly increasing or the edge multiset differs from its reverse (edges
 * compared with their weights through two independent 64-bit hash sums).
 * On success *out owns a default workspace for BFS and SSSP.
 */
gr_status gr_graph_create_csr(int32_t n, int64_t m, const int32_t* row_offsets,
                              const int32_t* cols, const uint32_t* weights, uint32_t flags,
                              void* stream, gr_graph** out);

/* Destroy a graph and its default workspace (synchronises the device; graphs
 * are long-lived, workspaces of a server are not: see gr_workspace_destroy_async). */
gr_status gr_graph_destroy(gr_graph* g);

/* Sizes and flags of a graph; any output pointer may be NULL.  Host call. */
gr_status gr_graph_info(const gr_graph* g, int32_t* n, int64_t* m, uint32_t* flags,
                        int32_t* max_degree);

/* Operations for footprint queries and workspaces. */
#define GR_OP_BFS  1
#define GR_OP_SSSP 2

/*
 * Device bytes one query of `op` needs beyond the graph itself (the
 * workspace size).  Feeds admission control in the paper's footprint model
 * alpha*|E| + beta*|V| (Sec. 7, memory usage discussion).  Host call.
 */
gr_status gr_graph_footprint(const gr_graph* g, int32_t op, size_t* bytes_per_query);

/*
 * Per-query scratch (frontier queues, bitmaps, packed SSSP keys, counters,
 * status word).  `ops` is a mask of GR_OP_BFS | GR_OP_SSSP.  Synchronous.
 */
gr_status gr_workspace_create(const gr_graph* g, int32_t ops, gr_workspace** out);
/* Waits for the whole device, then releases the workspace. */
gr_status gr_workspace_destroy(gr_workspace* ws);

/*
 * Stream-ordered workspaces, for a server whose streams must keep running
 * while one of them releases memory: the buffers come from the device's
 * stream-ordered allocator (cudaMallocAsync) and are initialised on `stream`,
 * so the workspace is ready for work queued on `stream` after the call and
 * nothing waits for the device.  Work on other streams must be ordered after
 * `stream` by the caller (events).  gr_workspace_destroy_async releases it
 * with cudaFreeAsync on `stream`, after the work already queued there; the
 * caller must also order any other stream that used it before that point.
 * BC, CC and triangle scratch allocated on such a workspace is released with
 * cudaFree (which waits for the device).  gr_workspace_destroy_async on a
 * workspace from gr_workspace_create behaves as gr_workspace_destroy.
 */
gr_status gr_workspace_create_async(const gr_graph* g, int32_t ops, void* stream,
                                    gr_workspace** out);
gr_status gr_workspace_destroy_async(gr_workspace* ws, void* stream);

/*
 * Wait for `stream`, then read and clear the status word of `ws` (NULL = the
 * graph's default workspace).  Returns GR_OK or the first device-detected
 * error since the last call (GR_ERR_CAPACITY, GR_ERR_OVERFLOW,
 * GR_ERR_TIMEOUT).  Synchronous.
 */
gr_status gr_sync_status(const gr_graph* g, gr_workspace* ws, void* stream);

/*
 * Work counters of the last gr_bfs / gr_sssp run on a workspace (the
 * quantities behind the paper's traversal-throughput accounting, Sec. 7
 * "Measurement methodology"):
 *   levels:   BFS levels, or SSSP near/far steps, executed;
 *   edges:    column entries read (edges inspected; pull levels stop early);
 *   vertices: rows opened (frontier rows and edge chunks expanded, pull
 *             candidates scanned, far-pile entries re-examined);
 *   updates:  vertices discovered (BFS) or successful relaxations (SSSP).
 */
typedef struct gr_run_stats {
  int32_t levels;
  int32_t reserved;
  int64_t edges;
  int64_t vertices;
  int64_t updates;
} gr_run_stats;

/* Wait for `stream` and read the counters of `ws` (NULL = default).  Synchronous. */
gr_status gr_last_run_stats(const gr_graph* g, gr_workspace* ws, gr_run_stats* out, void* stream);

/* ---- operator state ---------------------------------------------------- */

/*
 * State of the BFS visit functor (Sec. 6.1: set depth and predecessor on
 * discovery).  All pointers are device pointers of n entries.
 *   depth: int32, -1 = unvisited.  pred: int32 or NULL.
 *   level: depth of the input frontier; discovered vertices get level + 1.
 */
typedef struct gr_bfs_state {
  int32_t* depth;
  int32_t* pred;
  int32_t level;
} gr_bfs_state;

/*
 * State of the SSSP relax functor (Alg. 1 Update_Label / Set_Pred).  The
 * label and predecessor of v live together in one packed 64-bit key
 *   key[v] = ((uint64_t)dist << 32) | (uint32_t)pred
 * so that one 64-bit atomicMin updates both consistently; the result is the
 * smallest (dist, pred) pair offered, i.e. the minimum-id tight predecessor.
 * Unreached: key = UINT64_MAX (dist UINT32_MAX, pred -1).
 *   threshold: near/far split point for GR_FILTER_NEAR_FAR (dist < threshold
 *   is near).
 */
typedef struct gr_sssp_state {
  uint64_t* key;
  uint32_t threshold;
} gr_sssp_state;

/* ---- advance (Sec. 4.1, Sec. 5.1) --------------------------------------- */

/* mode bits */
#define GR_V2V       0  /* output vertex ids                                    */
#define GR_V2E       1  /* output edge ids (positions in C)                     */
#define GR_PUSH      0  /* expand the neighbour lists of the input frontier     */
#define GR_PULL      2  /* input = candidate (unvisited) vertices; Alg. 2       */
#define GR_ORDERED   0  /* output in the canonical order of the degree scan     */
#define GR_UNORDERED 4  /* any order (faster, atomics for placement)            */
#define GR_IDEMPOTENT 8 /* BFS visit without atomics; duplicates allowed        */

/* functors fused into the operator (Sec. 5.3) */
#define GR_FN_NONE       0  /* plain expansion                                  */
#define GR_FN_BFS_VISIT  1  /* state = gr_bfs_state*                            */
#define GR_FN_SSSP_RELAX 2  /* state = gr_sssp_state*                           */

/*
 * One advance step: in (device int32[in_len]) -> out (device int32[out_cap]).
 *   in_len: host count of input items; if in_len_dev is not NULL the count
 *   is read on the device from *in_len_dev and in_len is its upper bound.
 *   out_len: device int64*, receives the number of items produced.  If that
 *   number exceeds out_cap, only out_cap items are written, *out_len still
 *   receives the full count and the status word records GR_ERR_CAPACITY.
 *
 * GR_FN_NONE + GR_PUSH: out is the concatenation, in input order, of each
 *   input vertex's neighbour list (V2V) or edge-id range (V2E); with
 *   GR_UNORDERED the same multiset in any order.  Output-balanced: every
 *   CTA writes an equal slice of the output (Sec. 5.1.3, load balance over
 *   the output frontier).
 * GR_FN_BFS_VISIT + GR_PUSH: for every edge (u, v) of the input, v with
 *   depth -1 gets depth = level + 1 and pred = u, and is emitted once
 *   (atomic claim); with GR_IDEMPOTENT the claim is a plain check-and-set
 *   and v may be emitted more than once (Sec. 5.2.1).  Output order is
 *   unspecified.  State must be gr_bfs_state*.
 * GR_FN_BFS_VISIT + GR_PULL: each input vertex v with depth -1 scans its
 *   row in order and takes the first neighbour u with depth == level as
 *   parent (Alg. 2 Reverse_Advance); activated vertices are emitted in input
 *   order.  Requires a GR_SYMMETRIC graph.
 * GR_FN_SSSP_RELAX + GR_PUSH: for every edge (u, v, w) of the input with
 *   dist(u) finite, atomicMin(key[v], pack(dist(u) + w, u)); every v whose
 *   distance strictly dropped is emitted (possibly more than once).  Needs
 *   weights.  A sum >= UINT32_MAX is dropped; if its target is still
 *   unreached the status word records GR_ERR_OVERFLOW.
 */
gr_status gr_advance(const gr_graph* g, const int32_t* in, int64_t in_len,
                     const int64_t* in_len_dev, int32_t mode, int32_t functor, const void* state,
                     int32_t* out, int64_t out_cap, int64_t* out_len, void* stream);

/* ---- filter (Sec. 4.2) -------------------------------------------------- */

#define GR_FILTER_EXACT_UNIQUE 0 /* first occurrence of each id in [0,n), input order */
#define GR_FILTER_CULL         1 /* inexact: every valid id at least once, no new ids  */
#define GR_FILTER_UNVISITED    2 /* ignore `in`: all v with depth -1, ascending        */
#define GR_FILTER_NEAR_FAR     3 /* stable split by dist < threshold (Sec. 5.1.5)      */
#define GR_FILTER_MULTISPLIT   4 /* stable split into 2..8 distance buckets            */

/*
 * State of GR_FILTER_MULTISPLIT, the near/far split of Sec. 5.1.5 with more
 * than two buckets: item v goes to bucket
 *   b(v) = 0 if dist(v) < base, else min(buckets - 1, (dist(v) - base) / delta),
 * dist(v) = key[v] >> 32 (the packed SSSP keys of gr_sssp_state).
 *   buckets in [2, 8]; delta >= 1; bucket_len: device int64[buckets], receives
 *   the number of items of every bucket.
 */
typedef struct gr_multisplit_state {
  const uint64_t* key;
  uint32_t base;
  uint32_t delta;
  int32_t buckets;
  int64_t* bucket_len;
} gr_multisplit_state;

/*
 * One filter step: in (device int32[in_len]) -> out (+ far for NEAR_FAR).
 * Items outside [0, n) are dropped by every mode.
 *   EXACT_UNIQUE: exact stream compaction (global scan and scatter).
 *   CULL: the inexact "uniquification" of Sec. 4.2 / Sec. 5.2.1: out holds
 *     every valid input id at least once and no id more often than the
 *     input does; order unspecified.
 *   UNVISITED: state = gr_bfs_state*; in is ignored (may be NULL);
 *     out = { v : depth[v] == -1 } ascending (Alg. 2
 *     GenerateUnvisitedFrontier).
 *   NEAR_FAR: state = gr_sssp_state*; near items (dist < threshold) go to
 *     out, the rest to far, both in input order.  far/far_cap/far_len are
 *     required for this mode only.
 *   MULTISPLIT: state = gr_multisplit_state*; out = the items of bucket 0 in
 *     input order, then bucket 1, ...; bucket_len[j] = the items of bucket j;
 *     out_len = their total.  Uses a temporary from the stream-ordered
 *     allocator (8 bytes per bucket and 4096 items).
 * Lengths/capacities behave as in gr_advance.  Scratch comes from the
 * graph's default workspace, so concurrent filters on one graph must use
 * distinct streams serialised by the caller.
 */
gr_status gr_filter(const gr_graph* g, const int32_t* in, int64_t in_len,
                    const int64_t* in_len_dev, int32_t mode, const void* state, int32_t* out,
                    int64_t out_cap, int64_t* out_len, int32_t* far, int64_t far_cap,
                    int64_t* far_len, void* stream);

/* ---- BFS (Sec. 6.1, Sec. 5.1.4) ----------------------------------------- */

#define GR_DIR_AUTO 0  /* direction-optimising push/pull (Alg. 2, Eq. 5-6)     */
#define GR_DIR_PUSH 1  /* push only                                            */
#define GR_DIR_PULL 2  /* pull whenever the graph allows it (testing)          */

typedef struct gr_bfs_opts {
  int32_t direction;     /* GR_DIR_*                                            */
  float do_a;            /* push -> pull when m_f > m_u * do_a (Eq. 5)          */
  float do_b;            /* pull -> push when m_f < m_u * do_b (Eq. 6)          */
  int32_t big_degree;    /* rows at least this long are split into edge chunks
                            shared by the whole grid, rows of 32 edges up to
                            this length are expanded 4 per warp, shorter rows
                            32 per warp (Sec. 5.1.2 classes); 0 = library
                            default (256)                                     */
  int32_t blocks_per_sm; /* persistent grid = blocks_per_sm * SMs; 0 = max    */
  uint32_t spin_limit;   /* grid-barrier wait budget in polls; 0 = default    */
  gr_workspace* ws;      /* NULL = the graph's default workspace              */
  int32_t* level_stats;  /* optional device int32[4*max_levels]: per level
                            (frontier size, 1 if pull, sum of the frontier's
                            degrees m_f, start time in ns after the kernel
                            started, so level 0's start shows the
                            initialisation); one more row (frontier 0)
                            records when the level loop ended            */
  int32_t max_levels;    /* capacity of level_stats in levels                 */
  int32_t max_blocks;    /* upper bound on the persistent grid's CTAs; 0 = none.
                            A query on a high-diameter graph (small frontiers,
                            latency-bound levels) loses little on a quarter
                            of the SMs, and several such queries on separate
                            streams then run side by side                   */
  int64_t bulk_edges;    /* push levels whose frontier has at least this many
                            edges run in bulk: the expansion only marks
                            unvisited targets in the next-frontier bitmap
                            (reductions without return values), then one
                            pass over that bitmap writes the depths and
                            builds the next frontier; smaller push levels
                            claim each target with an atomic as they go.
                            0 = default (2 n, at least 65536), < 0 =
                            never.  Results do not depend on it             */
} gr_bfs_opts;

/* Fill *o with the library defaults. */
void gr_bfs_opts_default(gr_bfs_opts* o);

/*
 * Breadth-first search from src: depth[v] = fewest edges on a path src -> v
 * (device int32[n]), pred[v] = a parent one level up (device int32[n] or
 * NULL).  One persistent kernel runs the whole level loop on the device
 * (no per-level host round trip, Sec. 5.3).  opts may be NULL.
 */
gr_status gr_bfs(const gr_graph* g, int32_t src, int32_t* depth, int32_t* pred,
                 const gr_bfs_opts* opts, void* stream);

/* ---- SSSP (Sec. 3 example, Alg. 1, Sec. 5.1.5, Sec. 6.2) ---------------- */

typedef struct gr_sssp_opts {
  uint32_t delta;        /* near/far bucket width; 0 = derived from the graph */
  int32_t big_degree;    /* as in gr_bfs_opts; 0 = library default (1024)     */
  int32_t blocks_per_sm; /* as in gr_bfs_opts                                  */
  uint32_t spin_limit;   /* as in gr_bfs_opts                                  */
  gr_workspace* ws;      /* NULL = the graph's default workspace              */
  int32_t* level_stats;  /* optional device int32[4*max_levels]: per step
                            (near rows, 1 if a SPLIT step, far-pile length,
                            start time in ns after the kernel started); one
                            more row (0, 0, 0, time) records when the step
                            loop ended, before the distances are unpacked  */
  int32_t max_levels;    /* capacity of level_stats in steps                  */
  int32_t bulk_rows;     /* near frontiers of at least this many rows (a row
                            of 32 or more edges counts as 4, an edge chunk of
                            a split row as 8) are relaxed in
                            bulk: atomics without return values plus a
                            label-change bitmap, then one pass over the bitmap
                            builds the next piles; smaller ones enqueue per
                            edge.  0 = default: 64 on a graph with a row of
                            1024 or more edges, else n / 64 (at least 4096);
                            < 0 = never                                      */
  int32_t max_blocks;    /* as in gr_bfs_opts                                  */
  int32_t levels;        /* buckets of the priority queue (Sec. 5.1.5): 0 =
                            default, the multi-level queue of 8 (the current
                            bucket and the 7 after it keep lists of their own,
                            filled by a multisplit of the far pile); 2 = the
                            two-level near/far queue.  Results do not depend
                            on it                                             */
} gr_sssp_opts;

void gr_sssp_opts_default(gr_sssp_opts* o);

/*
 * Single-source shortest paths from src over the graph's weights:
 * dist[v] = minimum path weight (device uint32[n], GR_INF_DIST if
 * unreachable), pred[v] = the smallest-id tight predecessor (device int32[n]
 * or NULL).  Label-correcting advance/filter iterations with a two-level
 * near/far priority queue; one persistent kernel.  Needs weights.  If some
 * reachable vertex's shortest distance is >= UINT32_MAX the status word
 * records GR_ERR_OVERFLOW (such vertices are left at GR_INF_DIST).
 */
gr_status gr_sssp(const gr_graph* g, int32_t src, uint32_t* dist, int32_t* pred,
                  const gr_sssp_opts* opts, void* stream);

/* ---- multi-source BFS (batched queries) --------------------------------- */

typedef struct gr_msbfs_opts {
  int32_t direction;  /* GR_DIR_AUTO, GR_DIR_PUSH or GR_DIR_PULL (pull needs a
                         GR_SYMMETRIC graph)                                   */
  float push_ratio;   /* AUTO: pull once the active vertices' degree sum
                         exceeds push_ratio * m                              */
  int32_t snapshot_levels; /* levels kept as per-level visit snapshots (depths
                         then written in one coalesced pass); a traversal
                         deeper than this writes later depths directly as
                         bits appear, with two snapshots in ping-pong.  0 =
                         as many as fit in 2 GB (at least 2)              */
} gr_msbfs_opts;

void gr_msbfs_opts_default(gr_msbfs_opts* o);

/*
 * k independent BFS runs from srcs[0..k) (HOST array, each in [0, n)),
 * computed together bit-parallel, 256 sources per pass: every vertex holds
 * one bit per source (the multi-frontier traversal the paper names as future
 * work, Sec. 8).  depth: device int32[k * n]; depth[i * n + v] is the BFS
 * depth of v from srcs[i] (-1 if unreachable), exactly as gr_bfs would
 * report it.  Synchronous (the level loop reads one counter per level).  The
 * first call on a graph allocates the graph's multi-source scratch
 * (about 100 * n bytes plus the snapshots: up to 2 GB, or two levels' worth
 * when that is more), kept until gr_graph_destroy.  Calls on one graph are
 * serialised by the library (a second caller blocks until the first has
 * returned); calls on different graphs run concurrently.
 */
gr_status gr_bfs_multi(const gr_graph* g, const int32_t* srcs, int32_t k, int32_t* depth,
                       const gr_msbfs_opts* opts, void* stream);

/* ---- batched jobs over many graphs -------------------------------------- */

/*
 * One BFS or SSSP query of a batch.  The tuning fields choose the per-level
 * strategy of the job (0 = library default): do_a / do_b are the push/pull
 * switch factors of Eq. 5-6, big_degree the row length from which a row is
 * split into edge chunks shared by the whole job, delta the near/far bucket
 * width of SSSP (Sec. 5.1.5).
 */
typedef struct gr_job {
  const gr_graph* g;
  int32_t op;        /* GR_OP_BFS or GR_OP_SSSP                                */
  int32_t src;       /* in [0, n)                                              */
  void* out;         /* device int32 depth[n] (BFS) or uint32 dist[n] (SSSP)   */
  int32_t* pred;     /* device int32[n] or NULL                                */
  float do_a, do_b;
  int32_t big_degree;
  uint32_t delta;
} gr_job;

typedef struct gr_batch_opts {
  int32_t cluster_size;    /* CTAs (on distinct SMs) that run one job together, 1..16;
                              default 8                                              */
  int32_t clusters_per_sm; /* cap on resident clusters per SM; 0 = occupancy maximum  */
  int32_t use_graph;       /* capture the launch once in a CUDA graph and replay it   */
  uint32_t spin_limit;     /* reserved for bounded waits; 0 = default                 */
} gr_batch_opts;

void gr_batch_opts_default(gr_batch_opts* o);

typedef struct gr_batch gr_batch;

/*
 * Prepare a batch: copies the job table to the device (sorted largest job
 * first), allocates one scratch slot per resident cluster (sized for the
 * largest graph), and with use_graph captures the launch in a CUDA graph.
 * Synchronous.  The graphs and output arrays must outlive the batch.  Every
 * job produces exactly what gr_bfs / gr_sssp produce for it.
 */
gr_status gr_batch_create(const gr_job* jobs, int32_t njobs, const gr_batch_opts* opts,
                          gr_batch** out);

/* Run every job of the batch in one persistent launch on `stream` (async). */
gr_status gr_batch_run(gr_batch* b, void* stream);

/* Wait for `stream`; copy per-job status codes (may be NULL); return the first error. */
gr_status gr_batch_status(gr_batch* b, int32_t* job_status, void* stream);

/* Resident clusters, cluster size and scratch bytes of a batch (host call). */
gr_status gr_batch_info(const gr_batch* b, int32_t* clusters, int32_t* cluster_size,
                        size_t* scratch_bytes);

gr_status gr_batch_destroy(gr_batch* b);

/* ---- betweenness centrality (Sec. 6.3) ----------------------------------- */

typedef struct gr_bc_opts {
  int32_t big_degree;    /* rows at least this long are shared by the grid as
                            edge chunks in both passes; 0 = default (256)     */
  int32_t blocks_per_sm; /* persistent grid = blocks_per_sm * SMs; 0 = max    */
  uint32_t spin_limit;   /* grid-barrier wait budget in polls; 0 = default    */
  gr_workspace* ws;      /* NULL = the graph's default workspace              */
} gr_bc_opts;

void gr_bc_opts_default(gr_bc_opts* o);

/*
 * Brandes' betweenness-centrality pass for one source (Sec. 6.3): a forward
 * BFS that counts shortest paths, then a backward pass over the BFS levels
 * that accumulates dependencies.  Outputs (device arrays of n entries, each
 * may be NULL, then kept in workspace scratch):
 *   depth[v]: BFS depth from src (-1 unreachable);
 *   sigma[v]: number of shortest src -> v paths (sigma[src] = 1, 0 when
 *     unreachable), exact 64-bit integers; a count above INT64_MAX records
 *     GR_ERR_OVERFLOW in the status word (and the counts are then invalid);
 *   delta[v]: the dependency of src on v, the sum over edges (v, w) with
 *     depth[w] = depth[v] + 1 of sigma[v] / sigma[w] * (1 + delta[w]), in
 *     double precision (the summation order is not fixed: results agree
 *     with a sequential evaluation to within rounding);
 *   bc[v] (accumulated): bc[v] += delta[v] for every v != src, so that calls
 *     for several sources on one array sum the betweenness centrality over
 *     ordered (source, target) pairs.
 * Works on directed graphs too (paths follow edge directions).  The first
 * call on a workspace allocates its BC scratch (about 40 bytes per vertex
 * plus 8 bytes per 32 edges), kept until the workspace is destroyed.  One
 * persistent kernel, asynchronous on `stream`.
 */
gr_status gr_bc(const gr_graph* g, int32_t src, int32_t* depth, int64_t* sigma, double* delta,
                double* bc, const gr_bc_opts* opts, void* stream);

/* ---- connected components (Sec. 6.4) ------------------------------------ */

typedef struct gr_cc_opts {
  int32_t big_degree;    /* rows at least this long are shared by the grid as
                            edge chunks in the first hooking pass; 0 = default
                            (1024)                                           */
  int32_t blocks_per_sm; /* persistent grid = blocks_per_sm * SMs; 0 = max    */
  uint32_t spin_limit;   /* grid-barrier wait budget in polls; 0 = default    */
  gr_workspace* ws;      /* NULL = the graph's default workspace              */
} gr_cc_opts;

void gr_cc_opts_default(gr_cc_opts* o);

/*
 * Connected-component labels of a GR_SYMMETRIC graph (Sec. 6.4: hooking on an
 * edge frontier filtered to the edges whose end points still carry different
 * labels, then pointer jumping, repeated until no such edge remains).
 *   comp: device int32[n]; comp[v] = the smallest vertex id of v's component
 *     (a canonical labelling: equal for two vertices exactly when a path joins
 *     them).
 *   num_components: device int32* or NULL; receives the number of components.
 * Returns GR_ERR_UNSUPPORTED for a graph created without GR_SYMMETRIC.  The
 * first call on a workspace allocates its CC scratch (about 8 bytes per edge
 * plus 2 KB per resident warp), kept until the workspace is destroyed.  One
 * persistent kernel, asynchronous on `stream`.
 */
gr_status gr_cc(const gr_graph* g, int32_t* comp, int32_t* num_components,
                const gr_cc_opts* opts, void* stream);

/* ---- segmented intersection (Sec. 4.3) and triangle counting (Sec. 6.6) -- */

/*
 * Segmented intersection: for every pair i of the two input frontiers a, b
 * (device int32[len] each, ids in [0, n)), the ids present in both neighbour
 * lists N(a[i]) and N(b[i]).  Needs a GR_SYMMETRIC graph (its rows are
 * validated as strictly increasing, i.e. sorted sets); GR_ERR_UNSUPPORTED
 * otherwise.  A pair whose ids are not in [0, n) counts as empty and records
 * GR_ERR_INVALID_ARG in the status word.
 *   counts: device int64[len] or NULL; counts[i] = |N(a[i]) & N(b[i])|.
 *   total: device int64 or NULL; the sum of the counts.
 *   out: device int32[out_cap] or NULL; the intersections in pair order,
 *     each ascending (the output frontier of Sec. 4.3).  Requires counts and
 *     out_len (device int64, receives the total even when it exceeds
 *     out_cap; only out_cap items are written).
 *   ws: workspace whose scratch is used (NULL = the graph's default); the
 *     first call allocates the offsets array (8 bytes per pair), grown as
 *     needed and kept until the workspace is destroyed.
 * Asynchronous on `stream`.
 */
gr_status gr_segmented_intersect(const gr_graph* g, const int32_t* a, const int32_t* b,
                                 int64_t len, int64_t* counts, int64_t* total, int32_t* out,
                                 int64_t out_cap, int64_t* out_len, gr_workspace* ws,
                                 void* stream);

/*
 * Triangle counting of a GR_SYMMETRIC graph by the forward algorithm of
 * Sec. 6.6: each undirected edge is kept once, oriented by the (degree, id)
 * order of its end points (toward the larger end, which keeps every
 * out-list short), and every triangle is then the common out-neighbour of
 * the two ends of exactly one kept edge, found by the segmented intersection
 * above.
 *   total: device int64; the number of triangles (each counted once).
 *   per_vertex: device int64[n] or NULL; per_vertex[v] = the number of
 *     triangles containing v (costs one atomic per triangle).
 * The first call on a workspace allocates its scratch (about 14 bytes per
 * edge), kept until the workspace is destroyed.  Asynchronous on `stream`.
 */
gr_status gr_triangle_count(const gr_graph* g, int64_t* total, int64_t* per_vertex,
                            gr_workspace* ws, void* stream);

/* ---- BFS without allocation --------------------------------------------- */

/*
 * The paper has no counterpart for this entry point; it exists for callers
 * that must not allocate device memory while they run a query: a callback of
 * a custom device allocator or memory pool (allocating there would re-enter
 * the allocator), a latency-critical thread that cannot afford the implicit
 * synchronisation cudaMalloc may cause, or a host runtime that owns all
 * device memory.  It runs the same persistent BFS as gr_bfs, but takes the
 * CSR directly (no gr_graph handle, which would allocate) and keeps every
 * scratch buffer in one statically sized __device__ array of about 13 MB
 * that each GPU loading this library reserves until the process exits.  The
 * call allocates nothing.
 *
 *   n, m, row_offsets, cols: a CSR as gr_graph_create_csr accepts it; it is
 *     NOT validated here (the caller guarantees validity).  Limits:
 *     n <= GR_STATIC_MAX_VERTICES and m <= GR_STATIC_MAX_EDGES, otherwise
 *     GR_ERR_CAPACITY is returned and nothing runs.
 *   flags: 0 or GR_SYMMETRIC (trusted: allows direction-optimising pull
 *     levels; must only be passed for symmetric graphs with sorted rows).
 *   depth, pred: outputs as in gr_bfs (pred may be NULL).
 *   status: device int32* or NULL; receives GR_OK or the device-detected
 *     error of this run (as gr_sync_status would report it) when the run ends.
 * Asynchronous on `stream`.  The first call on a device looks up the scratch
 * address (cudaGetSymbolAddress, which may load the module) and so must not
 * be made while `stream` is being captured.  All calls share the one
 * scratch array: every call clears its control block and status word first,
 * and calls whose kernels overlap on the GPU race, so serialise them (for
 * example, issue them on one stream).
 */
#define GR_STATIC_MAX_VERTICES (1 << 20)
#define GR_STATIC_MAX_EDGES    (1 << 25)
gr_status gr_bfs_static(int32_t n, int64_t m, const int32_t* row_offsets, const int32_t* cols,
                        uint32_t flags, int32_t src, int32_t* depth, int32_t* pred,
                        int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GR_H_ */
