/*
 * ffg.h -- C ABI of the GB300 (sm_103a) fitness-flow-graph library.
 *
 * The library computes the landscape-difficulty metric of "Benchmarking
 * optimization algorithms for auto-tuning GPU kernels" (Schoonhoven, van
 * Werkhoven, Batenburg; arXiv 2210.01465):
 *
 *   1. the fitness flow graph (FFG) of a discrete tuning space (Sec. VII-B):
 *      every valid configuration is a node, with a directed edge to every
 *      neighbour -- Hamming (Sec. III-B, Eq. 2) or adjacent-value (the
 *      restriction stated right after Eq. 2) -- whose fitness is strictly
 *      lower;
 *   2. PageRank centrality of every node on that graph (Sec. VII-B);
 *   3. the p-proportion of centrality C_p (Sec. VII-B, Eq. 3): the share of
 *      the centrality of all local minima held by minima within (1+p) of the
 *      optimal fitness.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers documented "device" must be CUDA device (or managed) memory of
 *    the current device; "host" pointers are ordinary host memory.  The
 *    caller owns every buffer.  The library never allocates device memory:
 *    scratch space is a caller-provided workspace whose size is reported by
 *    the matching *_workspace_bytes function.  A workspace must be 256-byte
 *    aligned and must not be used by two calls that can run concurrently.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it in order; the only host
 *    synchronisations are the documented scalar read-backs.
 *  - Every function returns an ffg_status.  On an error other than
 *    FFG_ERR_NOT_CONVERGED the contents of output buffers are unspecified.
 *    Argument errors are detected on the host before any work is enqueued.
 *  - All functions are thread-safe as long as their buffers are distinct.
 */
#ifndef FFG_H
#define FFG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FFG_MAX_PARAMS 16       /* parameters per space */
#define FFG_MAX_VALUES 1024     /* entries over all value lists of a space */
#define FFG_MAX_CONSTRAINTS 16  /* clauses per space */
#define FFG_MAX_P 32            /* thresholds per centrality call */

typedef enum {
    FFG_OK = 0,
    FFG_ERR_INVALID_ARG = 1,   /* a bad argument, detected on the host */
    FFG_ERR_OVERFLOW = 2,      /* a size or product does not fit the index types */
    FFG_ERR_CUDA = 3,          /* a CUDA runtime call failed (see ffg_last_error) */
    FFG_ERR_EMPTY = 4,         /* the space has no valid configuration / no minimum */
    FFG_ERR_NOT_CONVERGED = 5, /* max_iter reached; the ranks are still written */
    FFG_ERR_TIMEOUT = 6,       /* a bounded device-side wait expired: PageRank's
                                  barriers give up after 2 s in which no block of
                                  any PageRank kernel made progress */
    FFG_ERR_NO_MEMORY = 7      /* the workspace passed is too small */
} ffg_status;

typedef enum { FFG_HAMMING = 0, FFG_ADJACENT = 1 } ffg_nbh;
typedef enum { FFG_F64 = 0, FFG_F32 = 1 } ffg_prec;

/* Constraint clause kinds.  P(mask) is the product of the values of the
 * parameters whose bit is set in `mask` (1 for an empty mask). */
typedef enum {
    FFG_PROD_LE = 0,      /* P(mask_a) <= bound                  */
    FFG_PROD_GE = 1,      /* P(mask_a) >= bound                  */
    FFG_DIVIDES = 2,      /* P(mask_b) != 0 and P(mask_a) % P(mask_b) == 0 */
    FFG_PROD_LE_PROD = 3  /* P(mask_a) <= P(mask_b)              */
} ffg_constraint_kind;

typedef struct {
    int32_t kind;      /* ffg_constraint_kind */
    uint32_t mask_a;   /* bit i = parameter i takes part in the left product */
    uint32_t mask_b;   /* right product (FFG_DIVIDES, FFG_PROD_LE_PROD) */
    int32_t reserved;  /* must be 0 */
    int64_t bound;     /* FFG_PROD_LE / FFG_PROD_GE bound */
} ffg_constraint;

/* A search space X = S_1 x ... x S_n (Sec. III-B), all arrays in HOST memory.
 * Raw point r has digits d_i in row-major order (the last parameter varies
 * fastest): r = sum_i d_i * stride_i, stride_{n-1} = 1,
 * stride_i = stride_{i+1} * radix_{i+1}; its value in parameter i is
 * values[offset_i + d_i] with offset_i = radix_0 + ... + radix_{i-1}.
 * A raw point is a valid configuration iff every clause holds.
 * Limits: 1 <= n_params <= 16; radix_i >= 1; sum(radix) <= 1024;
 * 0 <= n_constraints <= 16; product of radices <= 2^31 - 1; for every clause
 * and product, prod over the mask of max|value| < 2^63 (else
 * FFG_ERR_OVERFLOW). */
typedef struct {
    int32_t n_params;
    const int32_t *radix;
    const int64_t *values;
    int32_t n_constraints;
    const ffg_constraint *constraints;
} ffg_space;

/* The fitness flow graph in DEVICE memory, buffers owned by the caller.
 * Node v (0 <= v < n_nodes) is the v-th valid raw point in ascending raw
 * order.  Edge u -> v iff v is a neighbour of u and key(v) < key(u), where
 * key(x) = f(x) if f(x) < fail_thr and +inf otherwise (failed points, Sec. V:
 * fitness 1e10; NaN counts as failed).  Both adjacency lists of every node
 * are sorted by ascending node id.
 *   out_ptr[n_nodes+1], out_idx[n_edges]  -- CSR of out-edges (int64 / int32)
 *   in_ptr[n_nodes+1],  in_idx[n_edges]   -- CSR of in-edges
 *   outdeg[n_nodes]                        -- out-degree (int32)
 *   node_raw[n_nodes]                      -- raw index of each node (int64)
 *   is_min[n_nodes]                        -- 1 iff not failed and outdeg == 0
 *                                             (local minimum, Sec. III-B)
 * n_raw, n_nodes, n_edges, n_minima and f_opt (best non-failed fitness,
 * +inf if every node failed) are host fields written by ffg_build_count. */
typedef struct {
    int64_t n_raw, n_nodes, n_edges, n_minima;
    int64_t *out_ptr;
    int32_t *out_idx;
    int64_t *in_ptr;
    int32_t *in_idx;
    int32_t *outdeg;
    int64_t *node_raw;
    uint8_t *is_min;
    double f_opt;
} ffg_graph;

/* ---- FFG construction (Sec. III-B neighbourhoods, Sec. VII-B graph) ---- */

/* Bytes of workspace that ffg_build_count / ffg_build_fill need for `space`
 * (0 if the space is invalid). */
size_t ffg_workspace_bytes(const ffg_space *space, ffg_nbh nbh);

/* Phase 1 of the build.  fitness_raw: DEVICE, n_raw doubles in raw order.
 * Validates the space, marks valid points, counts degrees.  Writes
 * g->n_raw, n_nodes, n_edges, n_minima, f_opt (host fields; the device
 * pointers of g are not touched) and also *n_nodes / *n_edges when those host
 * pointers are non-NULL.  Synchronises `stream` once to read the counts.
 * Keeps per-space state in `workspace` for ffg_build_fill.
 * FFG_ERR_EMPTY if no configuration is valid. */
ffg_status ffg_build_count(const ffg_space *space, const double *fitness_raw, ffg_nbh nbh,
                           double fail_thr, ffg_graph *g, int64_t *n_nodes, int64_t *n_edges,
                           void *workspace, size_t ws_bytes, void *stream);

/* Phase 2: writes every device array of g.  Must follow ffg_build_count with
 * the same space, fitness, nbh, fail_thr and workspace (untouched in
 * between); g's host fields must be those written by ffg_build_count.
 * Fully asynchronous. */
ffg_status ffg_build_fill(const ffg_space *space, const double *fitness_raw, ffg_nbh nbh,
                          double fail_thr, ffg_graph *g, void *workspace, size_t ws_bytes,
                          void *stream);

/* ---- batched construction: many spaces in a few launches ----
 * A build job: a space (HOST), its fitness (DEVICE, n_raw doubles), the
 * neighbourhood, the failure threshold and its graph (HOST struct; DEVICE
 * arrays).  Same graphs, bit for bit, as ffg_build_count + ffg_build_fill
 * per job.
 *
 * ffg_build_batch_count runs the count phase of every job (a handful of
 * launches over all jobs) and one read-back, and writes each graph's
 * n_raw, n_nodes, n_edges, n_minima and f_opt; FFG_ERR_EMPTY if a job has
 * no valid configuration (all sizes are written).  The caller then gives
 * every graph its arrays and calls ffg_build_batch_fill, which records them
 * in the workspace and fills every graph (synchronises `stream` once).
 * ffg_build_batch_rerun repeats both phases from the tables in the
 * workspace with launches only (no host work, no synchronisation: it can be
 * captured in a CUDA graph); it is meant for unchanged inputs.  A job whose
 * recomputed counts differ from the sizes of its arrays (its fitness
 * changed) is left untouched and marked: ffg_build_batch_query reads the
 * per-job status (FFG_OK or FFG_ERR_INVALID_ARG) into status_out (HOST,
 * n_jobs) and returns the worst.  The workspace (DEVICE, 256-byte aligned,
 * ffg_build_batch_workspace_bytes) and the plan must stay untouched between
 * the calls. */
typedef struct {
    const ffg_space *space;
    const double *fitness_raw;
    int32_t nbh, reserved;
    double fail_thr;
    ffg_graph *g;
} ffg_build_job;

typedef struct {
    int32_t n_jobs, reserved;
    int64_t total_raw, total_words, total_blocks, total_rows;
    void *tables[20]; /* device pointers into the workspace (internal) */
} ffg_build_batch;

size_t ffg_build_batch_workspace_bytes(const ffg_build_job *jobs, int32_t n_jobs);
ffg_status ffg_build_batch_count(const ffg_build_job *jobs, int32_t n_jobs, void *workspace,
                                 size_t ws_bytes, ffg_build_batch *plan, void *stream);
ffg_status ffg_build_batch_fill(const ffg_build_job *jobs, int32_t n_jobs, ffg_build_batch *plan,
                                void *stream);
ffg_status ffg_build_batch_rerun(const ffg_build_batch *plan, void *stream);
ffg_status ffg_build_batch_query(const ffg_build_batch *plan, int32_t *status_out, void *stream);

/* ---- PageRank (Sec. VII-B) ----
 * Column-stochastic matrix A[v,u] = 1/outdeg(u) for every edge u -> v, with
 * damping `damping`, uniform teleport, and the mass of nodes without
 * out-edges spread uniformly:
 *   x'[v] = damping * sum_{u -> v} x[u]/outdeg[u]
 *           + (damping * sum_{outdeg(u)=0} x[u] + 1 - damping) / n_nodes.
 * Starts from x = 1/n_nodes (or from `ranks` when init has FFG_INIT_RANKS;
 * it must then hold a positive vector summing to 1) and stops when
 * sum_v |x'[v] - x[v]| < tol, returning x'.  The dangling mass, the
 * residual and the normalising sum are exact 64-bit fixed-point sums
 * (quantum 2^-60) read as FP64, in both precisions.  FFG_F32 keeps ranks and
 * per-row sums in FP32 and also stops once the residual stops decreasing
 * (the FP32 rounding floor).  `ranks` (DEVICE, n_nodes floats or doubles per
 * `prec`) receives x' normalised to sum 1.
 * iters_out / residual_out (HOST) receive the iteration count and the last
 * residual; when both are NULL nothing is synchronised and the result is
 * read later with pagerank_query.  FFG_ERR_NOT_CONVERGED after max_iter.
 * max_iter lies in [1, FFG_MAX_ITER] (else FFG_ERR_INVALID_ARG): the
 * blocks of a solve count their barrier arrivals in 32 bits.
 * `init` is a set of flags: FFG_INIT_RANKS (warm start from `ranks`) and
 * FFG_INIT_LAYOUT (the workspace already holds this graph's edge layout from
 * pagerank_prepare, or from an earlier solve of the same graph with the same
 * workspace and precision; without it the solve builds the layout first). */
#define FFG_INIT_RANKS 1
#define FFG_INIT_LAYOUT 2
#define FFG_MAX_ITER 1000000

size_t pagerank_workspace_bytes(int64_t n_nodes, int64_t n_edges, ffg_prec prec);

/* Builds, in `workspace`, the edge layout that pagerank_solve streams: per
 * tile of 32 rows, one (offset, row mask) descriptor per distinct in-edge
 * offset src - dst, plus the tiles' cost prefix used to split them between
 * blocks.  It depends on the graph only, so several solves of one graph
 * (other damping factors, warm starts) pass FFG_INIT_LAYOUT and skip it.
 * Asynchronous. */
ffg_status pagerank_prepare(const ffg_graph *g, ffg_prec prec, void *workspace,
                            size_t ws_bytes, void *stream);

ffg_status pagerank_solve(const ffg_graph *g, double damping, double tol, int32_t max_iter,
                          ffg_prec prec, void *ranks, int init, void *workspace,
                          size_t ws_bytes, int32_t *iters_out, double *residual_out,
                          void *stream);

/* pagerank_solve for callers that cannot allocate device memory (for
 * example code running while another component owns the device memory, or
 * where cudaMalloc is not allowed or would synchronise the device).  The
 * paper has no counterpart; this is a convenience of this library.
 * Same arguments and results as pagerank_solve minus the workspace: the
 * scratch space is a file-scope device array of 8 MiB that every device
 * holds from the moment the library is loaded until the process exits.
 * Graphs whose pagerank_workspace_bytes exceeds 8 MiB are rejected with
 * FFG_ERR_NO_MEMORY (about 48,000 nodes at 20 in-edges per node in FP32).
 * Every call looks up the array's device address on the current device;
 * the first lookup on a device loads the library's device code there, so
 * make the first call on a device before any stream capture.  Every call shares the one
 * array (the parts that must start at zero are cleared by each call), so
 * calls that overlap on the GPU -- from other streams or host threads --
 * race and must be serialised by the caller.  Always synchronises `stream`
 * once and returns the solve's status; iters_out / residual_out may be
 * NULL.  FFG_INIT_LAYOUT is ignored (the layout is always rebuilt); other
 * unknown init bits give FFG_ERR_INVALID_ARG. */
ffg_status pagerank_solve_static(const ffg_graph *g, double damping, double tol,
                                 int32_t max_iter, ffg_prec prec, void *ranks, int init,
                                 int32_t *iters_out, double *residual_out, void *stream);

/* ---- the naive metric (Sec. VII-A) ----
 * For every local minimum x (is_min), the fraction of optimal fitness
 * f_opt / f(x), in ascending node order: frac (DEVICE, g->n_minima
 * doubles) and, if node is non-NULL, the node ids (DEVICE, n_minima int64).
 * The number of minima is g->n_minima.  FFG_ERR_EMPTY without minima.
 * workspace: DEVICE, 256-byte aligned, minima_workspace_bytes.
 * Asynchronous. */
size_t minima_workspace_bytes(int64_t n_nodes);
ffg_status minima_fraction(const ffg_graph *g, const double *fitness_raw, double *frac,
                           int64_t *node, void *workspace, size_t ws_bytes, void *stream);

/* ---- exact solve on the DAG (Sec. VII-B) ----
 * The FFG has no cycles (every edge goes to a strictly better key), so
 *   y[v] = 1 + damping * sum_{u -> v} y[u] / outdeg[u]
 * is solved exactly in one pass over the nodes in topological order, level
 * by level: a level is the set of nodes whose in-neighbours are all done;
 * there are (longest improving path + 1) levels.  FP64, each in-list summed
 * in CSR order with one rounding per operation, so y does not depend on the
 * schedule.  Modes:
 * - FFG_DAG_VALUES: ranks = y, damping in [0, 1];
 * - FFG_DAG_PAGERANK: ranks = y / sum y, damping in (0, 1): the exact
 *   PageRank, the fixed point that pagerank_solve iterates towards;
 * - FFG_DAG_ABSORB: damping must be 1; ranks = y / n_nodes, the probability
 *   that a walk from a uniformly random node, moving to a uniformly random
 *   better neighbour, passes each node; at the nodes without out-edges
 *   (minima, and failed points without a better valid neighbour) the
 *   probability of ending there, which sum to 1.  Their C_p is
 *   centrality_proportion with FFG_F64.
 * Needs the out-edges as well as the in-edges.  ranks: DEVICE, n_nodes
 * doubles.  levels_out (HOST, may be NULL): the number of levels; when
 * non-NULL the call synchronises `stream` and reports FFG_ERR_TIMEOUT if a
 * bounded device wait expired.  workspace: DEVICE, dag_workspace_bytes. */
typedef enum { FFG_DAG_VALUES = 0, FFG_DAG_PAGERANK = 1, FFG_DAG_ABSORB = 2 } ffg_dag_mode;

size_t dag_workspace_bytes(int64_t n_nodes);
ffg_status dag_solve(const ffg_graph *g, double damping, ffg_dag_mode mode, double *ranks,
                     void *workspace, size_t ws_bytes, int32_t *levels_out, void *stream);

/* ---- simulated improving walks (Sec. VII-B) ----
 * A random walk on the FFG mimics a randomised first-improvement local
 * search.  walk_simulate runs n_walks walks: walk j starts at a uniformly
 * random node and moves to a uniformly random out-neighbour until it reaches
 * a node without out-edges; counts[v] (DEVICE, n_nodes uint64, overwritten)
 * = walks that ended at v.  Walk j's k-th draw (k = 0 for the start) is the
 * k-th output of the SplitMix64 stream whose state starts at
 * splitmix64(seed ^ j); a draw x picks index ((x >> 32) * m) >> 32 among m
 * choices.  The counts are reproducible bit for bit, and their expectation
 * is n_walks times dag_solve's FFG_DAG_ABSORB.  workspace: DEVICE, 256-byte
 * aligned, walk_workspace_bytes().  steps_out (HOST, may be NULL): moves
 * made; when non-NULL the call synchronises `stream` and reports
 * FFG_ERR_INVALID_ARG if a walk made n_nodes moves (a graph with a cycle;
 * impossible on an FFG; such a walk stops uncounted). */
size_t walk_workspace_bytes(void);
ffg_status walk_simulate(const ffg_graph *g, uint64_t seed, int64_t n_walks, uint64_t *counts,
                         void *workspace, size_t ws_bytes, int64_t *steps_out, void *stream);

/* ---- PageRank over a range of rows: the row-partitioned solve ----
 * The iteration of pagerank_solve (Sec. VII-B) split by rows, for a graph
 * shared by several ranks: a rank owns rows [row0, row1) and, per iteration,
 * forms w' of its rows from w of every row, where w = x / outdeg per row (x
 * for rows without out-edges).  Between iterations the ranks exchange their
 * rows of w' (an all-gather) and add their sums (an all-reduce); that host
 * side is paper_2210_01465_gb300.multi.  w is stored per row in
 * pagerank_rows_w_bytes(prec) opaque bytes (FFG_F32: a float; FFG_F64: an
 * exact 128-bit fixed-point value, so that a row-partitioned FP64 solve
 * equals pagerank_solve's bit for bit).
 *
 * pagerank_rows_workspace_bytes reads in_ptr[row0] and in_ptr[row1] from
 * the device (synchronously) and returns the range's workspace size (0 on
 * bad arguments).  pagerank_rows_prepare lays out the range's in-edges
 * (the same tiles and descriptors as pagerank_prepare, their offsets taken
 * from the global row); it also reads those two values.
 *
 * pagerank_rows_run enqueues one operation on the range (no host read, no
 * synchronisation).  `sums` (DEVICE, 4 uint64, added to): [0] residual
 * sum |x' - x|, [1] dangling mass, [2] sum of x, each fixed point with
 * quantum 2^-60, and [3] the number of bounded waits that expired.  `ctl`
 * (DEVICE, one ffg_rows_ctl, caller-owned) carries the solve's state
 * between operations; the decisions are taken there, on the device, from
 * the summed fixed-point values, with the arithmetic of pagerank_solve, so
 * that the host only moves bytes and reads ctl->stop.  w_in, w_out:
 * DEVICE, n_nodes w elements each (every row; w_out's rows of the range
 * are written).  ranks: DEVICE, n_nodes reals of the precision.
 *   FFG_ROWS_INIT:    w_out from x0 = ranks (or 1/n_nodes when NULL);
 *                     sums[1]; resets ctl.
 *   FFG_ROWS_STEP:    w_out = one iteration on w_in with `damping` and the
 *                     dangling mass in ctl; sums[0], sums[1], sums[3].
 *   FFG_ROWS_SUM:     sums[2] from w_in.
 *   FFG_ROWS_WRITE:   ranks = x * ctl->scale from w_in.
 * and three operations on ctl and the sums of every rank (after their
 * all-reduce), which also clear the sums they consume:
 *   FFG_ROWS_START:   ctl->dangling = sums[1] (after INIT).
 *   FFG_ROWS_ADVANCE: after a STEP: ctl->iters + 1, ctl->residual =
 *                     sums[0] / 2^60, ctl->dangling = sums[1]; ctl->stop
 *                     and ctl->converged when the residual is below `tol`
 *                     or (FFG_F32) stops decreasing, ctl->stop alone at
 *                     `max_iter`; ctl->status FFG_ERR_TIMEOUT (and stop)
 *                     if sums[3] is not 0.
 *   FFG_ROWS_SCALE:   ctl->scale = 1 / (sums[2] / 2^60) (after SUM).
 * The START, ADVANCE and SCALE launches are one thread each; with several
 * ranges in one process run them once, not per range. */
typedef enum {
    FFG_ROWS_INIT = 0, FFG_ROWS_STEP = 1, FFG_ROWS_SUM = 2, FFG_ROWS_WRITE = 3,
    FFG_ROWS_START = 4, FFG_ROWS_ADVANCE = 5, FFG_ROWS_SCALE = 6
} ffg_rows_kind;

typedef struct {               /* DEVICE; read by the host, written by the ops */
    int32_t iters, stop, converged, status;
    double residual, prev_residual, scale;
    uint64_t dangling;
} ffg_rows_ctl;

typedef struct {
    int32_t op;            /* ffg_rows_kind */
    int32_t max_iter;      /* ADVANCE */
    double damping;        /* STEP */
    double tol;            /* ADVANCE */
    const void *w_in;
    void *w_out;
    void *ranks;
    uint64_t *sums;
    ffg_rows_ctl *ctl;
} ffg_rows_op;

size_t pagerank_rows_w_bytes(ffg_prec prec);
size_t pagerank_rows_workspace_bytes(const ffg_graph *g, int64_t row0, int64_t row1,
                                     ffg_prec prec);
ffg_status pagerank_rows_prepare(const ffg_graph *g, int64_t row0, int64_t row1, ffg_prec prec,
                                 void *workspace, size_t ws_bytes, void *stream);
ffg_status pagerank_rows_run(const ffg_graph *g, int64_t row0, int64_t row1, ffg_prec prec,
                             const ffg_rows_op *op, void *workspace, size_t ws_bytes,
                             void *stream);

/* ---- batched PageRank: many solves in one persistent launch ----
 * A job is one PageRank solve (same definition and stopping rules as
 * pagerank_solve): graph g (host struct with DEVICE arrays), damping, tol,
 * max_iter, init (FFG_INIT_RANKS or 0), and `ranks` (DEVICE output, n_nodes
 * elements of the batch precision).  Jobs may share a graph (e.g. a damping
 * sweep): its edge layout is built once per run.  The batch form of the
 * survey shape of Sec. VII-B (one metric per kernel x GPU space). */
typedef struct {
    const ffg_graph *g;
    double damping, tol;
    int32_t max_iter, init;
    void *ranks;
} ffg_pr_job;

/* Filled by pagerank_batch_plan; plain data owned by the caller (device
 * pointers point into the plan's workspace).  A batch of at most
 * FFG_PR_PARAM_JOBS jobs also carries its job table in `params`, which
 * pagerank_batch_run passes to the kernel as its parameters (30 KB). */
#define FFG_PR_PARAM_JOBS 240
typedef struct {
    int32_t prec, n_jobs, n_graphs, n_blocks, warps, n_items, claim;
    int32_t w_form;  /* FP64: 1 = w kept as exact fixed point, 0 = as double */
    int64_t total_tiles;
    void *jobs, *graphs, *items, *first, *queue, *ctl;
    int64_t total_rows;
    void *tables[10]; /* per-row and per-tile tables of all graphs (internal) */
    int32_t param_jobs, reserved; /* jobs in `params` (n_jobs or 0) */
    uint64_t params[FFG_PR_PARAM_JOBS * 16]; /* the job table (internal) */
} ffg_pr_batch;

size_t pagerank_batch_workspace_bytes(const ffg_pr_job *jobs, int32_t n_jobs, ffg_prec prec);

/* Host-side planning: validates the jobs, gives every job a group of blocks
 * of one cooperative grid (large jobs several blocks, up to the whole grid;
 * small ones one) and an order:
 * - per-block lists: a job's ranks go to the least loaded blocks; every
 *   block runs its multi-block ranks in one global order (largest job
 *   first), then its one-block jobs (longest first onto the least loaded
 *   block), so a group only waits for blocks busy with an earlier job;
 * - claim order: every job's ranks as consecutive items, longest job
 *   first; a block takes the next unclaimed item whenever it is free, and a
 *   group starts when its last rank is taken.
 * Carves the workspace and uploads the tables.  Synchronises `stream`. */
ffg_status pagerank_batch_plan(const ffg_pr_job *jobs, int32_t n_jobs, ffg_prec prec,
                               void *workspace, size_t ws_bytes, ffg_pr_batch *plan,
                               void *stream);

/* Planning options.  A job whose cost exceeds `split` times the per-block
 * share of the batch gets its own blocks, about one per `grain` shares (the
 * others run on one block each); `max_blocks` caps the grid (0 = every
 * co-resident block); `block_warps` is 8 (256-thread blocks, several per SM),
 * 16 (one 512-thread block per SM, 128 registers per thread) or 24 (one
 * 768-thread block per SM), 0 = 24 for a batch of at most FFG_PR_PARAM_JOBS
 * jobs (its job table then travels in the kernel's parameters), else 16;
 * `claim` 1 selects the claim order, 0 the per-block lists; `fp64_form`
 * (FFG_F64 only) keeps w as exact 128-bit fixed point (1) or as double (2),
 * 0 = fixed point when every graph has at most 2^21 nodes; `min_tiles`
 * caps a job's group so that each warp of it has at least that many tiles
 * per iteration (0 or 1: one tile; larger values keep medium jobs on fewer
 * blocks, where the per-iteration barrier would cost more than the work it
 * spreads).  `job_cost` (HOST, n_jobs positive finite
 * values in any one unit, or NULL) replaces the cost model (edges + 20 x
 * nodes, times an iteration estimate from the damping) that sizes the groups
 * and balances the blocks, e.g. with the block-seconds that
 * pagerank_batch_times measured on an earlier run; it is read during the
 * call only.  pagerank_batch_plan uses 0.05, 0.005, 0, 0, 0, 0, 0, NULL.
 * They change only the schedule, never results or the workspace size. */
typedef struct {
    double split, grain;
    int32_t max_blocks, block_warps, claim, fp64_form, min_tiles, reserved;
    const double *job_cost;
} ffg_pr_tuning;

ffg_status pagerank_batch_plan_tuned(const ffg_pr_job *jobs, int32_t n_jobs, ffg_prec prec,
                                     const ffg_pr_tuning *tuning, void *workspace,
                                     size_t ws_bytes, ffg_pr_batch *plan, void *stream);

/* Enqueues the whole batch: the edge layout of every distinct graph (a few
 * launches over all of them) and one persistent launch that runs every job
 * to its own convergence.  Host work is argument checking only, so the
 * call can be captured in a CUDA graph and replayed (the graphs' contents
 * may change between replays, not their sizes or addresses).
 * pagerank_batch_prepare enqueues the layout step alone and
 * pagerank_batch_solve the solve alone; a solve needs the layout of the
 * graphs' current contents, from a prepare or an earlier run of the same
 * plan.  Run = prepare + solve. */
ffg_status pagerank_batch_run(const ffg_pr_batch *plan, void *stream);
ffg_status pagerank_batch_prepare(const ffg_pr_batch *plan, void *stream);
ffg_status pagerank_batch_solve(const ffg_pr_batch *plan, void *stream);

/* Per-job iterations, residuals and statuses (HOST arrays of n_jobs, each
 * may be NULL) of the last run; synchronises `stream`.  Returns FFG_OK if
 * every job converged, else the first non-OK status (FFG_ERR_TIMEOUT
 * first). */
ffg_status pagerank_batch_query(const ffg_pr_batch *plan, int32_t *iters_out,
                                double *residual_out, int32_t *status_out, void *stream);

/* Per-job busy time of the last run (a scheduling aid for the batched form
 * of Sec. VII-B's survey; the paper has no counterpart): block_seconds_out
 * (HOST, n_jobs) receives, for every job, the sum over its blocks of the
 * time each spent on it, from the moment all of them had started it to the
 * block's end of it (device global timer).  The total over the jobs, divided by the
 * plan's n_blocks, is the time an ideally balanced schedule would take.
 * Synchronises `stream`. */
ffg_status pagerank_batch_times(const ffg_pr_batch *plan, double *block_seconds_out,
                                void *stream);

/* Reads the outcome of the last pagerank_solve run in `workspace`
 * (synchronises `stream`).  Returns that run's status. */
ffg_status pagerank_query(const void *workspace, int32_t *iters_out, double *residual_out,
                          void *stream);

/* ---- proportion of centrality (Sec. VII-B, Eq. 3) ----
 * For each p[k] (HOST, 0 <= p[k], fractions such as 0.05, n_p <= 32):
 *   C_p = sum_{v min, f(v) <= thr_k} x[v] / sum_{v min} x[v],
 *   thr_k = f_opt * (1 + p[k]) evaluated in FP64 on the host.
 * fitness_raw is the build's DEVICE fitness; ranks is the DEVICE output of
 * pagerank_solve in precision `prec`.  Sums are compensated FP64.
 * cp_out (HOST, n_p doubles).  Synchronises `stream` once.
 * FFG_ERR_EMPTY if the graph has no local minimum. */
size_t centrality_workspace_bytes(int32_t n_p);

ffg_status centrality_proportion(const ffg_graph *g, const double *fitness_raw,
                                 const void *ranks, ffg_prec prec, const double *p,
                                 int32_t n_p, double *cp_out, void *workspace, size_t ws_bytes,
                                 void *stream);

/* Batched C_p: the same quantity for n_jobs graphs at once.  Job j: g (host
 * struct with DEVICE arrays), fitness_raw and ranks (DEVICE, precision
 * `prec`).  f_opt is taken on the device as the smallest fitness of a
 * local minimum (the global optimum is one, and no minimum is failed, so it
 * equals the build's f_opt), and thr_k = f_opt * (1 + p[k]) is formed there
 * with the same two FP64 roundings; the host fields f_opt / n_minima of g
 * are not read, so a graph rebuilt on the device needs no new plan.
 *
 * centrality_batch_plan uploads the job table and p into `workspace`
 * (DEVICE, centrality_batch_workspace_bytes(n_jobs, n_p), 256-byte
 * aligned) and fills `plan` (plain data owned by the caller; synchronises
 * `stream` once).  centrality_batch_run enqueues the computation -- a reset
 * and three launches, no host work beyond argument checks, so it can be
 * captured in a CUDA graph -- and writes plan->cp (DEVICE, n_jobs x n_p
 * doubles, row-major) and plan->status (DEVICE, per job FFG_OK, or
 * FFG_ERR_EMPTY when the graph has no local minimum: its row is NaN).
 * centrality_batch_query synchronises `stream` and copies them to cp_out /
 * status_out (HOST, each may be NULL); it returns FFG_ERR_EMPTY if any job
 * is empty.  centrality_batch does all three (cp_out required). */
typedef struct {
    const ffg_graph *g;
    const double *fitness_raw;
    const void *ranks;
} ffg_cp_job;

typedef struct {
    int32_t n_jobs, n_p, prec, reserved;
    double *cp;        /* DEVICE results, n_jobs x n_p (in the workspace) */
    int32_t *status;   /* DEVICE per-job status (in the workspace) */
    void *tables[8];   /* device pointers into the workspace (internal) */
} ffg_cp_batch;

size_t centrality_batch_workspace_bytes(int32_t n_jobs, int32_t n_p);

ffg_status centrality_batch_plan(const ffg_cp_job *jobs, int32_t n_jobs, ffg_prec prec,
                                 const double *p, int32_t n_p, void *workspace,
                                 size_t ws_bytes, ffg_cp_batch *plan, void *stream);
ffg_status centrality_batch_run(const ffg_cp_batch *plan, void *stream);
ffg_status centrality_batch_query(const ffg_cp_batch *plan, double *cp_out,
                                  int32_t *status_out, void *stream);

ffg_status centrality_batch(const ffg_cp_job *jobs, int32_t n_jobs, ffg_prec prec,
                            const double *p, int32_t n_p, double *cp_out, void *workspace,
                            size_t ws_bytes, void *stream);

/* ---- a whole batch in one call (Sec. VII-B over many search spaces) ----
 * ffg_batch_run re-runs a batch planned with the calls above, in order on
 * `stream`:
 *   1. every FFG (ffg_build_batch_rerun of `build`; skipped when NULL,
 *      e.g. when the graphs are built once and only the dampings vary);
 *   2. every PageRank solve (pagerank_batch_run of `pagerank`);
 *   3. C_p of every job of `cp` at its fractions (centrality_batch_run;
 *      skipped when NULL).  Its jobs normally pair each PageRank job's graph
 *      and ranks with the graph's fitness, in the PageRank plan's precision.
 * With out == NULL the three steps are only enqueued: no host work beyond
 * argument checks, no synchronisation, so the call can be captured in a
 * CUDA graph (the results stay in device memory: the plans' cp / status
 * arrays and the PageRank job outputs).  Otherwise the call synchronises
 * `stream` and fills every non-NULL field of `out` (HOST arrays):
 * build_status (one per build job; FFG_ERR_INVALID_ARG marks a job whose
 * recomputed sizes no longer fit its arrays, which keeps its previous
 * graph), iters / residual / pr_status (one per PageRank job) and cp
 * (cp->n_jobs x cp->n_p, row-major; needs `cp`).  The plans, the workspaces
 * and every buffer they name belong to the caller and must stay valid.
 * Returns the worst status: FFG_ERR_CUDA or FFG_ERR_TIMEOUT first, else the
 * first of the build, PageRank (FFG_ERR_NOT_CONVERGED) and C_p
 * (FFG_ERR_EMPTY: a graph without a local minimum, its row NaN) statuses;
 * FFG_ERR_INVALID_ARG for a missing or empty plan, or out->cp without `cp`
 * (nothing launched). */
typedef struct {
    const ffg_build_batch *build;  /* from ffg_build_batch_count + _fill, or NULL */
    const ffg_pr_batch *pagerank;  /* from pagerank_batch_plan(_tuned); required */
    const ffg_cp_batch *cp;        /* from centrality_batch_plan, or NULL */
} ffg_batch_desc;

typedef struct {
    int32_t *build_status;         /* HOST, one per build job, or NULL */
    int32_t *iters;                /* HOST, one per PageRank job, or NULL */
    double *residual;              /* HOST, one per PageRank job, or NULL */
    int32_t *pr_status;            /* HOST, one per PageRank job, or NULL */
    double *cp;                    /* HOST, cp->n_jobs x cp->n_p, or NULL */
} ffg_batch_out;

ffg_status ffg_batch_run(const ffg_batch_desc *desc, ffg_batch_out *out, void *stream);

/* ---- diagnostics ---- */
const char *ffg_status_str(ffg_status s);
/* Detail of the last error raised on the calling thread ("" if none). */
const char *ffg_last_error(void);
/* Number of kernels this library has launched in this process. */
uint64_t ffg_launch_count(void);
/* Bounds-checked builds (compiled with -DFFG_CHECKED): every index a kernel
 * derives from caller data -- CSR entries, row pointers, layout descriptors
 * -- is checked before the access it guards; a failed check skips the
 * access and is counted.  ffg_checked_build returns 1 in such a build, 0
 * otherwise.  ffg_checked_failures returns the number of failed checks since
 * the last reset (0 in a normal build), stores the site code of the first
 * one in *first_code (if non-NULL; 0 if none) and, when `reset` is non-zero,
 * clears the record.  Site codes: 1xx PageRank (101 a gather outside w, 102
 * a layout write outside the tile's room), 2xx FFG build (201/202 a CSR
 * write or a node id outside the node's row or the nodes,
 * 203 a neighbour outside the raw points), 3xx DAG solve (301 an
 * out-neighbour, 302 an in-neighbour outside the nodes), 401 a walk step
 * to a node outside the nodes, 5xx C_p (501 in the rank sums, 502 in the
 * minima listing: a node's raw point outside the fitness). */
int ffg_checked_build(void);
uint64_t ffg_checked_failures(uint64_t *first_code, int reset);

#ifdef __cplusplus
}
#endif
#endif /* FFG_H */
