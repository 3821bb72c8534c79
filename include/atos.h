/*
 * atos.h -- C ABI of a GB300 (sm_103a) task-parallel dynamic scheduler for irregular graph work.
 *
 * The library implements the scheduling model of "Atos: A Task-Parallel GPU Dynamic Scheduling
 * Framework for Dynamic Irregular Computations" (Chen et al., PPoPP 2022): one device-wide
 * worklist of vertex tasks, popped by warp- or CTA-sized workers in a persistent kernel (or one
 * discrete launch per queue generation), with a tunable fetch size (Sections 3 and 4, Listing 2
 * and the launch API of Listing 3).  Three relaxed-dependency applications run on it (Section 5):
 * speculative BFS (Algorithm 2), asynchronous push-residual PageRank (Algorithm 4) and
 * speculative greedy colouring (Algorithm 6); the level-synchronous forms (Algorithms 1, 3, 5) are
 * available as the BSP comparator.
 *
 * Conventions for every entry point:
 *   - Graphs are undirected int32 CSR: row_ptr[n + 1] (row_ptr[0] = 0, non-decreasing,
 *     row_ptr[n] = nnz) and col[nnz] with 0 <= col[k] < n; each undirected edge appears in both
 *     rows.  nnz must fit in int32.
 *   - Output buffers are DEVICE memory allocated by the caller (for example torch tensors);
 *     small control arrays (BFS sources) are HOST memory.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work is stream-ordered.
 *   - Return value: ATOS_OK (0) or a negative ATOS_ERR_* code.  No C++ exception crosses the ABI.
 *     When a call is given a non-NULL `stats`, it synchronises `stream`, fills `stats` and returns
 *     the device-side status as well (for example ATOS_ERR_QUEUE_OVERFLOW); with stats == NULL
 *     it returns once the work is enqueued and reports only host-side errors.
 *   - Calls on one graph object share its scratch memory: do not let two calls on the same graph
 *     object overlap on the device.  Different graph objects are independent.
 *   - The library owns the memory it allocates and frees it in atos_graph_destroy /
 *     atos_batch_destroy.
 */
#ifndef ATOS_H_
#define ATOS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define ATOS_OK 0
#define ATOS_ERR_INVALID_ARG (-1)    /* NULL pointer, size out of range, bad config */
#define ATOS_ERR_BAD_CSR (-2)        /* row_ptr not monotone, col out of range, not symmetric */
#define ATOS_ERR_OOM (-3)            /* device allocation failed */
#define ATOS_ERR_QUEUE_OVERFLOW (-4) /* a worklist ring ran out of slots; results are invalid */
#define ATOS_ERR_TIMEOUT (-5)        /* a device-side wait exceeded spin_limit_ns */
#define ATOS_ERR_CUDA (-6)           /* a CUDA runtime call failed (no device, launch error...) */
#define ATOS_ERR_UNSUPPORTED (-7)    /* configuration not built (e.g. this worker size) */
#define ATOS_ERR_BUSY (-8)           /* serving: no free slot or not enough arena memory now */
#define ATOS_ERR_BOUNDS (-9)         /* bounds-checked builds only: an index outside its array was
                                        caught (and the access redirected) during the run */

/* ------------------------------------------------------------------ configuration */
#define ATOS_WORKER_WARP 32 /* worker_size == 32: one warp per worker (persist-32) */
#define ATOS_WORKER_THREAD 1 /* worker_size == 1: one thread per worker, scheduled per warp (the
                                warp pops up to fetch_size <= 32 tasks, each lane runs one; a task
                                whose row exceeds 32 entries is run by the whole warp); every
                                application and batches (servers pause CTA workers only) */

#define ATOS_PERSISTENT 0 /* one launch; workers loop on the queue until it drains (Section 3.4) */
#define ATOS_DISCRETE 1   /* one launch per queue generation; the host reads the next size */
#define ATOS_BSP 2        /* level-synchronous comparator (Algorithms 1, 3, 5) */

#define ATOS_FETCH_FIXED 0  /* every pop reserves exactly fetch_size slots */
#define ATOS_FETCH_GREEDY 1 /* a pop reserves min(fetch_size, tasks available), at least 1 */
#define ATOS_FETCH_SPREAD 2 /* a pop reserves min(fetch_size, available / workers), at least 1 */

/* atos_config.flags */
#define ATOS_FLAG_PHANTOM_TASK 1u /* test hook: count one task that is never pushed, so that the
                                     workers wait for it until spin_limit_ns and report
                                     ATOS_ERR_TIMEOUT (exercises the bounded waits) */
#define ATOS_FLAG_PR_CROSSING 2u  /* PageRank: a push that lifts a neighbour's residue from <= eps to
                                     > eps enqueues that neighbour (threshold crossing), in place of
                                     the Check_Size scan of Algorithm 4 (Section 5.2).  Same fixed
                                     point and the same final verification sweep; check_size is
                                     ignored.  Persistent and discrete strategies; BSP ignores it. */

#define ATOS_FLAG_SPREAD_IDS 4u   /* PageRank and colouring (persistent and discrete strategies) run on
                                     an internal copy of the graph with its vertices renamed, built on
                                     the device at the first such call (4 (2 n + 1) + 4 nnz bytes; the
                                     build synchronises the stream once).  The highest-degree vertices
                                     (whole degree classes, at most 16384 and n / 32) take ids that
                                     are multiples of 32 (one per 128-byte line), spread over the id
                                     range; the rest are spread over the remaining ids by the
                                     bijection r -> (a r + c) mod m (a ~ 0.618 m, coprime to m).  On
                                     scale-free graphs sorted rows all begin with the few low-id hubs,
                                     so a warp's 32 state updates land in a few L2 slices; spread ids
                                     balance them over the slices, and PageRank's CTA workers add the
                                     updates bound for the hubs in shared memory, sending each hub one
                                     update per batch.  Results come back in the caller's ids (one
                                     gather).  Batches and servers apply it to their PageRank and
                                     colouring instances, and the BSP strategy to its PageRank and
                                     colouring; BFS ignores it. */

#define ATOS_FLAG_USE_TUNED 8u     /* atos_bfs / atos_pagerank / atos_color use the configuration
                                     cached by atos_autotune for the graph's class (all fields),
                                     or this one without the flag when the class is not tuned */

#define ATOS_FLAG_GC_ORDERED 16u   /* colouring: an assign task avoids only the colours of the vertex's
                                     smaller-id neighbours (in the ids the run uses); the check tasks
                                     are unchanged, so a conflict with a larger neighbour still makes
                                     that neighbour recolour.  The result stays proper and follows
                                     first fit in id order closely: fewer colours on scale-free
                                     graphs (Algorithm 6's assign considers every neighbour) */

#define ATOS_FLAG_BFS_EXPAND_ONCE 32u /* BFS (atos_bfs, persistent and discrete): a vertex queued
                                     several times is expanded once per depth.  A task first
                                     records its depth in a per-vertex marker (atomicMin) and skips
                                     the expansion if a copy of the vertex popped after the same
                                     improvement already expanded it.  Removes nearly all of the
                                     asynchronous BFS's re-expansions on scale-free graphs, at one
                                     atomic per task (n int32 per source of scratch). */

#define ATOS_FLAG_BSP_DEVICE_LOOP 64u /* ATOS_BSP: the level loop runs on the device: each level's
                                     kernels are the body of a CUDA graph whose conditional WHILE node
                                     repeats them until the next frontier is empty (one graph launch
                                     per call, no host synchronisation per level).  Without it the host
                                     reads the next frontier's size after every level. */

#define ATOS_FLAG_BSP_PER_SOURCE 128u /* ATOS_BSP BFS: one source after another.  Without it the
                                     frontiers of a group of sources advance together, one launch of
                                     each level kernel per level for the whole group: cfg->window
                                     sources (0 = as many as keep their depth arrays within about
                                     64 MB, half of L2, as the persistent strategy's window). */

#define ATOS_FLAG_GC_DEPENDENCY 256u /* atos_color (persistent and discrete strategies): colour each
                                     vertex once, after all of its smaller-id neighbours (in the ids
                                     the run uses), with the smallest colour none of them holds: a
                                     per-vertex count of uncoloured smaller neighbours makes a vertex
                                     ready, and the task that colours a vertex sets its colour in a
                                     bitmap of each larger neighbour and counts the neighbour down, so
                                     a ready vertex reads only its own bitmap.  The result is exactly
                                     serial first fit in id order, one task per vertex and no
                                     recolouring; the run takes as many dependent steps as the longest
                                     path of increasing ids.  With a CTA worker, rows with more than
                                     2080 larger neighbours are counted down partly by other CTAs
                                     (segment tasks of 2048 entries).  Scratch, per vertex layout and
                                     built on first use: the rows split at the smaller neighbours
                                     (n + nnz int32), the bitmaps (n int2 + about n + nnz / 64 words),
                                     the segment table (16 bytes per possible segment), and n int32
                                     counts.  The BSP strategy ignores it; batches and servers return
                                     ATOS_ERR_UNSUPPORTED. */

#define ATOS_FLAG_BFS_SPLIT_ROWS 512u /* atos_bfs with a CTA worker (worker_size >= 64, persistent
                                     and discrete): a popped vertex whose row holds more than 8192
                                     entries is pushed back as segment tasks of 4096 entries, which
                                     any worker expands, instead of one CTA walking the whole row.
                                     A segment re-reads the vertex's depth when it runs and is
                                     dropped if the vertex has improved since (the copy queued by the
                                     improvement expands the row).  About 2 nnz / 4096 16-byte table
                                     entries per source of scratch; when the table is full a row is
                                     expanded whole.  Ignored by other workers, batches and servers. */

typedef struct atos_config {
  int32_t worker_size;    /* 1 (thread worker), 32 (warp worker) or a CTA worker of 64,
                             128, 256, 512 or 1024 threads */
  int32_t fetch_size;     /* tasks per pop, 1..1024; at most worker_size for CTA workers (FETCH_SIZE
                             of Section 4); at most 32 for thread and warp workers */
  int32_t strategy;       /* ATOS_PERSISTENT, ATOS_DISCRETE or ATOS_BSP */
  int32_t fetch_policy;   /* ATOS_FETCH_FIXED, _GREEDY or _SPREAD (persistent strategy only) */
  int32_t num_blocks;     /* persistent grid size; 0 = all CTAs that fit at once (occupancy x SMs) */
  int32_t check_size;     /* PageRank: vertex ids checked per task (Check_Size of Algorithm 4);
                             0 = 32 */
  int32_t window;         /* batched runs: instances active at once; 0 = automatic (also the
                             group size of a multi-source BSP BFS) */
  uint32_t flags;         /* ATOS_FLAG_* */
  int64_t queue_capacity; /* ring slots per instance, rounded up to a power of two; 0 = automatic */
  int64_t spin_limit_ns;  /* budget of any single device-side wait; 0 = 4 seconds */
} atos_config;

/* Per-call statistics (filled when the call is given a non-NULL pointer). */
typedef struct atos_stats {
  double ms;              /* device time of the call's kernels (CUDA events on `stream`) */
  int64_t tasks;          /* tasks popped and processed, summed over instances */
  int64_t edges;          /* neighbour entries read by task bodies */
  int64_t pushes;         /* tasks pushed (children, re-checks, re-colourings) */
  int64_t iterations;     /* kernel launches of the scheduling loop (1 when persistent) */
  double residual_l1;     /* PageRank: FP64 sum of the residues left (unnormalised scale) */
  double error_bound;     /* PageRank: bound on the L1 distance of the normalised result to the
                             normalised fixed point, from an FP64 a-posteriori certificate:
                             ||(1 - alpha) 1 + alpha P x - x||_1 / ((1 - alpha) S) for the
                             result scaled to the fixed point's sum S = n - alpha * (isolated
                             vertices); it covers the FP32 rounding of the ranks */
  int32_t num_colors;     /* colouring: colours used */
  int32_t status;         /* device-side status (ATOS_OK or ATOS_ERR_*) */
  int64_t batches;        /* worker batches that processed at least one task (tasks / batches is
                             the mean batch; 0 for the BSP strategy) */
  int64_t idle_polls;     /* pops of persistent workers that found nothing to run */
} atos_stats;

typedef struct atos_graph_s* atos_graph_t;

/* atos_graph_create flags */
#define ATOS_DEVICE_PTRS 1u      /* row_ptr and col are device pointers */
#define ATOS_BORROW 2u           /* with ATOS_DEVICE_PTRS: use the caller's buffers in place; the
                                    caller keeps them alive and unchanged until destroy */
#define ATOS_CHECK_SYMMETRIC 4u  /* also verify that every entry (u, v) has its mirror (v, u) */
#define ATOS_SKIP_VALIDATION 8u  /* trust the CSR: skip the monotonicity, column-range and symmetry
                                    checks; row_ptr[0] == 0 and row_ptr[n] == nnz are still checked */

/* ------------------------------------------------------------------ entry points */

/* Fills *cfg with the preset named `preset`: NULL or "default" (persistent CTA worker of 256
 * threads, fetch 256), "persist-warp" (Section 6.2's persist-32), "persist-cta", "discrete-cta",
 * "discrete-warp", "bsp", or "autotune" (the defaults plus ATOS_FLAG_USE_TUNED: each call takes
 * the configuration atos_autotune cached for its graph's class and application, and the
 * defaults when there is none).  Returns ATOS_ERR_INVALID_ARG for an unknown name or NULL cfg. */
int atos_queue_config(atos_config* cfg, const char* preset);

/* Host-side CSR check (the one atos_graph_create runs on host pointers).  flags may contain
 * ATOS_CHECK_SYMMETRIC.  Returns ATOS_OK, ATOS_ERR_INVALID_ARG (NULL pointer, n < 0, nnz < 0 or
 * nnz > INT32_MAX) or ATOS_ERR_BAD_CSR.  Touches no GPU. */
int atos_csr_validate(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, uint32_t flags);

/* Uploads (or, with ATOS_DEVICE_PTRS | ATOS_BORROW, adopts) an undirected CSR graph of n
 * vertices and nnz entries (the CSR of Section 5's algorithms: vertex.neighbors /
 * neighborLen).  Host CSR is validated on the host.  Device CSR: row_ptr is copied to the host
 * and checked there, every column index is range-checked by a kernel (which only compares it),
 * and ATOS_CHECK_SYMMETRIC runs on a host copy of col.  ATOS_SKIP_VALIDATION keeps only the
 * row_ptr[0] == 0 and row_ptr[n] == nnz checks: the caller then vouches for the CSR.
 * On success *out receives a handle owned by the caller until atos_graph_destroy.  n == 0 is
 * allowed (an empty graph). */
int atos_graph_create(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, uint32_t flags,
                      void* stream, atos_graph_t* out);

/* Frees everything the library allocated for g (synchronises the device first).  NULL is a
 * no-op. */
int atos_graph_destroy(atos_graph_t g);

/* Reports the vertex count, entry count and maximum degree of g (any pointer may be NULL). */
int atos_graph_info(atos_graph_t g, int32_t* n, int64_t* nnz, int32_t* max_degree);

/* Breadth-first search from each of nsrc sources (Section 5.1; Algorithm 2 when the strategy is
 * persistent or discrete, Algorithm 1 for ATOS_BSP, whose levels cover every source's frontier
 * at once unless ATOS_FLAG_BSP_PER_SOURCE).  sources: HOST array of nsrc vertex ids in
 * [0, n).  depths: DEVICE int32 array of nsrc * n entries, row s = hop distances from
 * sources[s], INT32_MAX for vertices outside the source's component.  All nsrc searches run in
 * one launch with one worklist each (cfg->window of them active at a time).  Errors:
 * ATOS_ERR_INVALID_ARG for a NULL pointer, nsrc < 1 or a source out of range. */
int atos_bfs(atos_graph_t g, const int32_t* sources, int32_t nsrc, int32_t* depths, const atos_config* cfg,
             void* stream, atos_stats* stats);

/* Push-residual PageRank (Section 5.2; Algorithm 4 persistent or discrete, Algorithm 3 for
 * ATOS_BSP) on the unnormalised scale of the paper: rank starts at 1 - alpha, the residue
 * of v starts at (1 - alpha) alpha sum_{u in N(v)} 1 / deg(u), and a task pushes
 * alpha * residue / deg(v) to each neighbour.  Runs until every residue is at most eps.  rank:
 * DEVICE float array of n entries, returned normalised to sum 1 (the sum is taken in FP64).
 * alpha in (0, 1), eps > 0.  The FP64 residual and error bound are reported in stats. */
int atos_pagerank(atos_graph_t g, float alpha, float eps, float* rank, const atos_config* cfg, void* stream,
                  atos_stats* stats);

/* Speculative greedy colouring (Section 5.3; Algorithm 6's task uberkernel, Algorithm 5 for
 * ATOS_BSP): every vertex takes the smallest colour not held by a neighbour, then re-checks;
 * of two adjacent vertices with the same colour the one with the larger id recolours.  colors:
 * DEVICE int32 array of n entries, each in [0, deg(v)], proper on termination.  num_colors:
 * HOST int32 receiving the number of colours used (may be NULL; filled after a stream sync). */
int atos_color(atos_graph_t g, int32_t* colors, int32_t* num_colors, const atos_config* cfg, void* stream,
               atos_stats* stats);

/* Diagnostics: after synchronising the device, copies the queue control words of the last
 * launch's first ninst instances on g (words[i]: tasks pushed in the high 32 bits, tasks
 * completed in the low 32 bits; heads[i]: pop tickets handed out) and the site of the first
 * device wait that ran out of budget (0 = none; 1 ring slot, 2 CTA worker idle, 3 warp worker
 * idle, 4 successor hand-over, 5 worker lifetime).  Any output pointer may be NULL.  Returns
 * ATOS_ERR_INVALID_ARG if ninst exceeds the instances g's scratch holds. */
int atos_debug_queue_state(atos_graph_t g, int32_t ninst, uint64_t* words, uint32_t* heads, int32_t* fail_site);

/* Diagnostics: after synchronising the device, counts the set bits of g's queued-vertex bitmap
 * (PageRank / colouring) and the occupied slots of its rings; after a successful run both are
 * zero.  Either pointer may be NULL. */
int atos_debug_scratch_check(atos_graph_t g, uint64_t* set_bits, uint64_t* busy_slots);

/* Diagnostics: the vertex layout of the spread-id copy of g (ATOS_FLAG_SPREAD_IDS), built first
 * if needed (which synchronises `stream`).  perm: HOST int32 array of n entries receiving the
 * copy's id of every vertex (may be NULL); *hubs (may be NULL) receives H, the number of hubs:
 * the vertices of the largest degree classes (four classes per power of two), whole classes while
 * they fit in min(16384, 2^k), 2^k the largest power of two <= n / 32, ranked by decreasing class
 * and increasing vertex id within a class.  The hub of rank i has the id 32 ((mul i + add) mod
 * 2^k) with mul odd: one hub per 128-byte line of a 4-byte state array, at most.  The other
 * vertices take the remaining ids in spread order. */
int atos_debug_spread_layout(atos_graph_t g, int32_t* perm, int32_t* hubs, void* stream);

/* Throughput timeline (tracing; the throughput-over-time view of Section 6.4, Figures 1-3): the
 * persistent and discrete calls on g that follow record, per bucket of bucket_ns nanoseconds
 * from the start of the call, the tasks and neighbour entries of the worker batches that ended
 * in it (the last bucket takes everything later).  nbuckets = 0 turns it off.  It costs two
 * global atomics per batch while on.  The BSP strategy records nothing.  Synchronises the
 * device. */
int atos_timeline(atos_graph_t g, int64_t bucket_ns, int32_t nbuckets);

/* The timeline of the last call on g: tasks[b] and edges[b] (HOST arrays of nbuckets, the
 * configured count; either may be NULL).  Synchronises the device. */
int atos_timeline_read(atos_graph_t g, int64_t* tasks, int64_t* edges, int32_t nbuckets);

/* Ceilings of the task bodies' edge loops on g, with no scheduler: one pass over every CSR
 * entry in order, a coalesced read of col[e] and then
 *   ATOS_CEILING_SCATTER: red.add.f32 into state[col[e]] (PageRank's residue scatter), or
 *   ATOS_CEILING_GATHER:  a load of state[col[e]] (BFS's and colouring's neighbour reads),
 * into an n-float scratch the call allocates.  *ms_per_pass: mean device time of one pass over
 * `repeats` passes after a warm-up pass (stream-ordered on `stream`, which it synchronises).
 * nnz / ms_per_pass is the edge rate those loops can reach on this graph: the roofline of
 * the PageRank kernel (on the input layout of an RMAT graph the sorted rows send a warp's
 * updates to few L2 slices; ATOS_CEILING_SPREAD_IDS measures the spread layout). */
#define ATOS_CEILING_SCATTER 0
#define ATOS_CEILING_GATHER 1
#define ATOS_CEILING_SPREAD_IDS 2 /* or-ed into kind: measure on the spread-id copy of the graph
                                     (the layout ATOS_FLAG_SPREAD_IDS runs on; built if needed) */
int atos_edge_ceiling(atos_graph_t g, int32_t kind, int32_t repeats, double* ms_per_pass, void* stream);

/* The library keeps the device and pinned host blocks of destroyed graphs, batches and servers
 * for reuse by later ones of the same sizes.  This returns every cached block to the driver
 * (*cached_bytes_before, may be NULL, receives how many bytes were cached). */
int atos_pool_trim(int64_t* cached_bytes_before);

/* Number of CUDA kernels this library has launched in this process (monotone counter, all
 * threads, all devices); lets a caller count the launches of a region of its own program. */
uint64_t atos_kernel_launches(void);

/* ------------------------------------------------------------------ batched launches */

#define ATOS_APP_BFS 0
#define ATOS_APP_PAGERANK 1
#define ATOS_APP_COLOR 2

/* One instance of a batch: an application on one of the batch's graphs. */
typedef struct atos_instance {
  int32_t app;    /* ATOS_APP_BFS, ATOS_APP_PAGERANK or ATOS_APP_COLOR */
  int32_t graph;  /* index into the graphs array given to atos_batch_create */
  int32_t source; /* BFS: source vertex */
  float alpha;    /* PageRank: damping in (0, 1) */
  float eps;      /* PageRank: residue threshold > 0 (unnormalised scale) */
  int32_t reserved;
  void* out;      /* DEVICE output of n entries: int32 depths (BFS), float ranks summing to 1
                     (PageRank) or int32 colours (colouring); owned by the caller */
} atos_instance;

typedef struct atos_batch_s* atos_batch_t;

/* Creates a batch of ninst instances over ngraphs graphs (extension of the paper's single queue
 * to one worklist per instance; Section 3's scheduler, several problems at once).  Everything a
 * run needs (instance table, rings, control blocks, PageRank and colouring scratch) is
 * allocated here; the graphs and output buffers must stay alive until atos_batch_destroy.
 * cfg: persistent or discrete strategy (ATOS_ERR_UNSUPPORTED for BSP); with the persistent one
 * cfg->window instances are active at a time (0 = as many as fit in about half of L2); the
 * discrete one launches each queue generation of every instance at once.  Errors: ATOS_ERR_INVALID_ARG for
 * NULL pointers, ninst outside [1, 65535], a bad graph index, source, alpha or eps. */
int atos_batch_create(const atos_graph_t* graphs, int32_t ngraphs, const atos_instance* inst, int32_t ninst,
                      const atos_config* cfg, atos_batch_t* out);

/* Enqueues one run of every instance on `stream`.  Persistent strategy: stream-ordered kernel
 * launches and memsets only (no host synchronisation, no allocation), so the call can be captured
 * in a CUDA graph.  Discrete strategy: the host loop synchronises `stream` after every generation.
 * Calls on one batch must not overlap on the device. */
int atos_batch_run(atos_batch_t b, void* stream);

/* Same as atos_batch_run, but the first call captures the run into a CUDA graph (on a private
 * stream) and every call replays it with one graph launch on `stream`.  Persistent strategy only
 * (ATOS_ERR_UNSUPPORTED for a discrete batch, whose generations the host drives). */
int atos_batch_run_graph(atos_batch_t b, void* stream);

/* Synchronises `stream` and reports the last run: *total sums the instances' counters (ms = the
 * run's device time); per_instance (ninst entries, may be NULL) gets each instance's counters,
 * PageRank residual_l1 and error_bound (the FP64 certificate of the returned ranks, as for
 * atos_pagerank) and colouring num_colors.  Returns the device status of the run. */
int atos_batch_stats(atos_batch_t b, atos_stats* total, atos_stats* per_instance, void* stream);

/* Instances, active window and persistent grid size of a batch (any pointer may be NULL). */
int atos_batch_info(atos_batch_t b, int32_t* ninst, int32_t* window, int32_t* grid);

/* Frees a batch (synchronises the device first).  NULL is a no-op. */
int atos_batch_destroy(atos_batch_t b);

/* ------------------------------------------------------------------ serving */

/* Completion record of a served request. */
typedef struct atos_completion {
  int64_t id;          /* the id atos_server_submit returned */
  int32_t status;      /* ATOS_OK or the device status of the epoch that ended the request */
  int32_t app;         /* ATOS_APP_* */
  int32_t graph;
  int32_t num_colors;  /* colouring */
  int64_t tasks;       /* tasks processed for this request */
  int64_t edges;       /* neighbour entries read for this request */
  int64_t epochs;      /* server epochs run so far (when the request completed) */
  double error_bound;  /* PageRank: FP64 certificate of the returned ranks (see atos_stats) */
} atos_completion;

typedef struct atos_server_s* atos_server_t;

/* A request server over resident graphs (continuous batching).  max_slots: requests in flight
 * at most; budget_bytes: device memory for the requests' scratch (ring, pending tickets,
 * PageRank residues, queued bits), allocated first-fit per request and released at completion.
 * cfg: persistent CTA workers only (ATOS_ERR_UNSUPPORTED otherwise).  Graphs must outlive the
 * server. */
int atos_server_create(const atos_graph_t* graphs, int32_t ngraphs, int32_t max_slots, int64_t budget_bytes,
                       const atos_config* cfg, atos_server_t* out);

/* Admits a request if a slot is free and its scratch fits in the arena now (else ATOS_ERR_BUSY,
 * nothing changed) and initialises its state on the server's stream; it runs from the next
 * atos_server_step on.  req->out is the caller's DEVICE output (as in atos_instance), written
 * when the request completes.  *id receives the request id. */
int atos_server_submit(atos_server_t s, const atos_instance* req, int64_t* id);

/* Runs one epoch: one persistent launch over every admitted request, in which each worker
 * pauses at a safe point once slice_ns have passed (0 = 1 ms) and leaves the tickets it holds to
 * the next epoch.  Requests that terminated are finished (PageRank normalised, colours counted),
 * their completion records queued and their slots and memory released.  Synchronises the
 * server's stream.  *active_left (may be NULL) receives the requests still in flight.  A lap of
 * a request's ring must take longer than a slice (rings hold at least 2^20 slots). */
int atos_server_step(atos_server_t s, int64_t slice_ns, int32_t* active_left);

/* Moves up to max queued completion records to out; *count receives how many. */
int atos_server_poll(atos_server_t s, atos_completion* out, int32_t max, int32_t* count);

/* Requests in flight, arena bytes in use and in total, epochs run (any pointer may be NULL). */
int atos_server_info(atos_server_t s, int32_t* active, int64_t* arena_used, int64_t* arena_size, int64_t* epochs);

/* Frees a server (synchronises the device first).  NULL is a no-op. */
int atos_server_destroy(atos_server_t s);

/* ------------------------------------------------------------------ autotuning */

/* PageRank candidates of atos_autotune whose reported FP64 error bound (atos_stats.error_bound,
 * L1 distance of the normalised result to the fixed point) exceeds this are not chosen. */
#define ATOS_TUNE_PR_MAX_ERROR 1e-4

/* Colouring candidates of atos_autotune whose colour count exceeds this factor times the fewest
 * colours any candidate reached are not chosen. */
#define ATOS_TUNE_GC_MAX_COLOR_RATIO 1.05

/* Times candidate configurations of `app` (ATOS_APP_*) on g and returns the fastest in *best
 * (its device time in *best_ms): CTA workers of 128..1024 threads, warp workers and thread
 * workers, fixed / greedy / spread fetch policies, persistent, discrete and BSP strategies (the
 * BSP level loop on the host and on the device), plus the instance window, expansion markers
 * and row splitting for BFS, Check_Size and the threshold-crossing enqueue for PageRank, and the dependency-ordered mode
 * for colouring (Figure 4's worker-size x FETCH_SIZE sweep with the kernel strategy of
 * Section 3.4).  Each candidate runs repeats + 1 times (the first warms up); failing candidates,
 * PageRank candidates whose error bound exceeds ATOS_TUNE_PR_MAX_ERROR and colouring candidates
 * with more than ATOS_TUNE_GC_MAX_COLOR_RATIO times the fewest colours are skipped.  sources/nsrc: BFS
 * sources (HOST).
 * scratch_out: DEVICE output buffer the runs write into (nsrc * n int32 for BFS, n floats for
 * PageRank, n int32 for colouring).  The winner is cached per graph class (application, log2 n,
 * log2 average degree, log2 max/average degree).  Synchronises `stream`. */
int atos_autotune(atos_graph_t g, int32_t app, const int32_t* sources, int32_t nsrc, void* scratch_out,
                  int32_t repeats, atos_config* best, double* best_ms, void* stream);

/* Autotuner for a batch: creates the batch under each candidate configuration -- CTA workers of
 * 128..1024 threads and warp workers, fetch policies, instance windows, the persistent strategy
 * (replayed as a CUDA graph) and the discrete one, and PageRank's threshold-crossing enqueue --
 * runs it repeats + 1 times (the first warms up) and returns the fastest in *best (device time of
 * one run in *best_ms).  Candidates that fail, or whose largest PageRank error bound exceeds
 * ATOS_TUNE_PR_MAX_ERROR, are skipped.  Arguments as for atos_batch_create; outputs are written
 * by the runs.  Synchronises `stream`. */
int atos_batch_autotune(const atos_graph_t* graphs, int32_t ngraphs, const atos_instance* inst, int32_t ninst,
                        int32_t repeats, atos_config* best, double* best_ms, void* stream);

/* The configuration cached by atos_autotune for g's graph class and `app`: ATOS_OK, or
 * ATOS_ERR_UNSUPPORTED (and the defaults in *cfg) when that class has not been tuned. */
int atos_tuned_config(atos_graph_t g, int32_t app, atos_config* cfg);

/* ------------------------------------------------------------------ allocation-free BFS */

/* Largest graph atos_bfs_noalloc accepts (its fixed ring holds 2^20 slots, the floor atos_bfs
 * gives a single search). */
#define ATOS_NOALLOC_MAX_VERTICES 262144

/* Single-source BFS (same result as atos_bfs) that allocates no memory, for callers that must
 * not call cudaMalloc: code living inside an application whose own allocator owns the device
 * memory, plug-ins forbidden to allocate, or latency-critical loops that cannot pay the device
 * synchronisation an allocation may imply.  The paper has no counterpart of this entry point.
 *   row_ptr, col: DEVICE int32 CSR of an undirected graph (n + 1 and nnz entries), unchanged
 *   during the call; source in [0, n); depth: DEVICE int32[n] receiving the hop distances
 *   (INT32_MAX outside the source's component).
 * The CSR is checked on the device before the search reads it (row_ptr[0] == 0, row_ptr[n] ==
 * nnz, rows non-decreasing, every column index in [0, n); symmetry is not checked), at the cost
 * of one host round trip; a malformed CSR returns ATOS_ERR_BAD_CSR and the search does not run.
 * Scratch: one fixed array of about 8.2 MiB of device memory inside the library image, held by
 * every GPU that loads the library until the process exits, and shared by all calls on that GPU.
 * Each call looks up the array's device address (cudaGetSymbolAddress) on the current device; the
 * first call on a device also initialises the array; make that first call before any stream
 * capture.  Calls that overlap on the GPU (other streams, other host threads) race on the shared
 * scratch and must be serialised by the caller.  The call synchronises `stream` and returns the
 * device status (ATOS_OK, ATOS_ERR_TIMEOUT, ATOS_ERR_QUEUE_OVERFLOW), ATOS_ERR_BAD_CSR or
 * ATOS_ERR_CUDA; it returns ATOS_ERR_INVALID_ARG for NULL pointers, a source out of range, nnz
 * outside [0, INT32_MAX], or n < 1 or n > ATOS_NOALLOC_MAX_VERTICES (checked before any GPU
 * work). */
int atos_bfs_noalloc(const int32_t* row_ptr, const int32_t* col, int32_t n, int64_t nnz, int32_t source,
                     int32_t* depth, void* stream);

/* Human-readable name of a status code (static storage). */
const char* atos_status_string(int status);

/* Library version string (static storage). */
const char* atos_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ATOS_H_ */
