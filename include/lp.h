/*
 * lp.h - C ABI of the GB300 (sm_103a) RAK label-propagation library.
 *
 * Method: RAK / LPA label propagation as used by Sahu, "Selecting a suitable
 * Parallel Label-propagation based algorithm for Disjoint Community
 * Detection" (arXiv 2301.09125).
 *   Sec. 3.2  every vertex starts with a unique label; in each iteration every
 *             vertex adopts the label carrying the most interconnecting edge
 *             weight among its neighbours; maximum-weight ties are broken by
 *             taking the first of them (strict) or a random one (non-strict);
 *             the run converges once at most a `tolerance` fraction of the
 *             vertices changed label in an iteration (0.05 recommended).
 *   Sec. 3.3  asynchronous update: a vertex may read labels its neighbours
 *             took earlier in the same iteration.
 *   Sec. 1    modularity (Newman-Girvan) scores the resulting partition.
 *   Sec. 3.1  graphs are undirected (every edge stored in both directions)
 *             and weighted.
 *
 * Conventions for every entry point:
 *   - Every call returns an lp_status and never aborts the process.  On
 *     failure lp_last_error() returns a message for the calling thread.
 *   - Graphs are CSR with int32 row offsets (n+1 entries, offsets[0] = 0,
 *     non-decreasing, offsets[n] = m), int32 column indices in [0, n) and
 *     int32 weights >= 1 (NULL = every weight is 1).  The CSR is used exactly
 *     as given: a stored entry (v,u,w) is A_vu = w; a stored self-loop counts
 *     the vertex's own label; duplicate entries add up.  The library does not
 *     symmetrise (LP_FLAG_CHECK_SYMMETRIC only checks).
 *   - The order of entries inside a row is significant: the strict tie rule
 *     picks, among the maximum-weight labels, the one whose first occurrence
 *     in the row comes first.
 *   - Non-strict ties: among the maximum-weight labels, the one with the
 *     smallest 64-bit key mix(mix(mix(seed + (t+1)G) + (v+1)G) + (l+1)G),
 *     where mix is the SplitMix64 output function (Steele, Lea & Flood 2014),
 *     G = 0x9E3779B97F4A7C15, t = iteration + iter_offset, v the vertex and l
 *     the label, both local to the graph; equal keys fall back to the strict
 *     rule.
 *   - Converged iff changed <= tolerance * n in double precision, where n
 *     counts every vertex (isolated ones keep their label and never count as
 *     changed).  Reaching max_iter first is not an error (converged = 0).
 *   - All device work is ordered on the CUDA stream given at creation time.
 *     Calls on one object are not thread-safe; distinct objects may be used
 *     from distinct threads.
 */
#ifndef LP_H
#define LP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LP_OK = 0,
    LP_EINVAL = 1,   /* bad argument or invalid CSR / labels */
    LP_ENOMEM = 2,   /* device or pinned host allocation failed */
    LP_ECUDA = 3,    /* a CUDA runtime call failed */
    LP_ETIMEOUT = 4, /* a bounded device-side wait ran out */
    LP_ENOTREADY = 5 /* no result yet (serving poll) */
} lp_status;

enum { LP_SYNC = 0, LP_ASYNC = 1 };

enum {
    LP_FLAG_DEVICE_PTRS = 1,     /* offsets/indices/weights are device pointers */
    LP_FLAG_CHECK_SYMMETRIC = 2, /* also reject a CSR whose pattern/weights are not symmetric */
    LP_FLAG_BORROW = 4           /* with DEVICE_PTRS: keep the caller's arrays instead of
                                    copying them (caller keeps them alive and unchanged
                                    until lp_graph_destroy); indices and weights that do
                                    not start on a 16-byte boundary are copied anyway */
};

/* Parameters of one RAK run (Sec. 3.2). */
typedef struct {
    double tolerance;           /* in [0, 1]; converged iff changed <= tolerance*n (default 0.05) */
    int32_t max_iter;           /* >= 1 (default 20) */
    int32_t mode;               /* LP_SYNC: every vertex reads the previous iteration's labels
                                   (double buffer).  LP_ASYNC: a vertex also reads labels
                                   written earlier in the same iteration (Sec. 3.3), in the
                                   wave order given by `waves`. */
    int32_t strict;             /* 1 = strict "first" tie rule, 0 = non-strict "random" */
    int32_t iter_offset;        /* added to the iteration index seen by the non-strict key
                                   (resume a run without changing its random stream) */
    uint64_t seed;              /* non-strict key seed */
    const int32_t *init_labels; /* NULL = unique labels label[v] = v (Sec. 3.2); else n
                                   labels in [0, n) (resume from lp_labels_get) */
    int32_t init_labels_on_device; /* 1 if init_labels is a device pointer */
    int32_t waves;              /* LP_ASYNC only: the order of in-place updates (Sec. 3.3
                                   leaves it open) is W >= 1 waves, wave(v) = v mod W (v local);
                                   waves run in order 0..W-1 and store their labels when the
                                   whole wave has chosen, so a vertex reads this iteration's
                                   label of a neighbour in an earlier wave and the previous
                                   iteration's label of any other.  W = 1 equals LP_SYNC;
                                   W >= n is plain in-place updating in ascending vertex order.
                                   Deterministic for every W.  Default 31; after clamping to
                                   the largest graph's n, W must be <= 4096. */
} lp_rak_params;

/* Outcome of one run. */
typedef struct {
    int32_t iterations;   /* iterations executed, including the one that met the test */
    int32_t converged;    /* 1 if the tolerance test was met, 0 if max_iter stopped it */
    int64_t last_changed; /* vertices that changed label in the last iteration */
    float gpu_ms;         /* device time of the iteration loop (CUDA events) */
} lp_rak_result;

typedef struct lp_graph lp_graph;

/* Fill *p with the defaults: tolerance 0.05 (Sec. 3.2), max_iter 20,
 * LP_SYNC, strict, iter_offset 0, seed 0, init_labels NULL, waves 31.
 * Errors: LP_EINVAL if p is NULL. */
lp_status lp_rak_params_default(lp_rak_params *p);

/* Ingest one graph (Sec. 3.1: undirected, weighted): validate the CSR, copy it
 * to the device (unless borrowed) and sort its vertices into degree buckets.
 *   n, m      vertex and stored-entry counts; 0 <= n, 0 <= m < 2^31.
 *   offsets   int32[n+1]; indices int32[m]; weights int32[m] or NULL.
 *             Host pointers unless flags has LP_FLAG_DEVICE_PTRS.  The caller
 *             keeps ownership; nothing is retained after return unless
 *             LP_FLAG_BORROW is given.
 *   flags     LP_FLAG_* bits.
 *   cuda_stream  cudaStream_t used for all work on this graph (NULL = the
 *             legacy default stream).
 *   out       receives the new graph handle.
 * Errors: LP_EINVAL for a NULL argument, n < 0, m out of range, offsets not a
 * row pointer, an index outside [0, n), a weight < 1, a vertex whose summed
 * weight is >= 2^31, or (with LP_FLAG_CHECK_SYMMETRIC) an asymmetric CSR;
 * LP_ENOMEM; LP_ECUDA.  On error *out is left NULL and nothing leaks. */
lp_status lp_graph_create(int32_t n, int64_t m, const int32_t *offsets, const int32_t *indices,
                          const int32_t *weights, uint32_t flags, void *cuda_stream,
                          lp_graph **out);

/* Free the graph and every device buffer it owns (NULL is a no-op). */
lp_status lp_graph_destroy(lp_graph *g);

/* Vertex and entry counts of a graph.  Errors: LP_EINVAL on NULL. */
lp_status lp_graph_info(const lp_graph *g, int32_t *n, int64_t *m);

/* Run RAK to convergence (Sec. 3.2; asynchronous variant Sec. 3.3).
 * The result labels stay on the device (lp_labels_get, lp_modularity).
 * Returns after the run has finished on the device.  A run that repeats the
 * previous run's parameters on the same graph is captured once as a CUDA
 * graph (on its first repeat) and replayed afterwards; runs whose waves all
 * take one cooperative launch per iteration (many waves, rows of at most 32
 * entries) are always launched from the host.  Results are the same either
 * way.
 * Errors: LP_EINVAL for NULL arguments, tolerance outside [0, 1],
 * max_iter < 1, mode not LP_SYNC/LP_ASYNC, waves < 1 or too large (LP_ASYNC),
 * init_labels outside [0, n);
 * LP_ENOMEM; LP_ECUDA. */
lp_status lp_rak_run(lp_graph *g, const lp_rak_params *p, lp_rak_result *out);

/* Number of vertices that changed label in each iteration of the last run.
 * Writes min(capacity, iterations) values to changed and the iteration count
 * to *count.  Errors: LP_EINVAL on NULL g or count, or changed NULL with
 * capacity > 0. */
lp_status lp_rak_history(const lp_graph *g, int64_t *changed, int32_t capacity, int32_t *count);

/* Copy the current labels (n int32 vertex ids) to dst, a host pointer unless
 * dst_on_device is 1.  Before any run the labels are the unique labels.
 * Errors: LP_EINVAL on NULL; LP_ECUDA. */
lp_status lp_labels_get(lp_graph *g, int32_t *dst, int32_t dst_on_device);

/* Modularity (Sec. 1) of a partition of the graph:
 *   Q = sum_c [ L_c / 2m - (K_c / 2m)^2 ]
 * with A the stored CSR, k_v = sum_u A_vu, 2m = sum_v k_v, L_c = sum of A_vu
 * over stored entries with both ends in c, K_c = sum of k_v over c.  L, K_c
 * and 2m are summed exactly in 64-bit integers and sum_c K_c^2 exactly in 128
 * bits; Q = L/2m - (sum_c K_c^2)/(2m)^2 is formed in double.  Q = 0 when the
 * graph has no entries.
 *   labels  n labels in [0, n) (host pointer unless labels_on_device), or NULL
 *           for the graph's current labels.
 * Errors: LP_EINVAL on NULL g/q or a label outside [0, n); LP_ENOMEM; LP_ECUDA. */
lp_status lp_modularity(lp_graph *g, const int32_t *labels, int32_t labels_on_device, double *q);

/* ---------------------------------------------------------------------------
 * Batches: many independent graphs in one device arena, iterated together.
 * Each graph keeps its own convergence test and iteration count; a graph that
 * has converged stops changing while the others continue.  Labels and vertex
 * ids are local to each graph.
 * ------------------------------------------------------------------------- */
typedef struct lp_batch lp_batch;

typedef struct {
    int32_t n;
    int64_t m;
    const int32_t *offsets; /* host int32[n+1] */
    const int32_t *indices; /* host int32[m] */
    const int32_t *weights; /* host int32[m] or NULL (unit) */
} lp_graph_desc;

/* Ingest `count` graphs (host CSR, validated as in lp_graph_create) into one
 * device arena.  flags: LP_FLAG_CHECK_SYMMETRIC only.
 * Errors: LP_EINVAL (bad count or any invalid graph; the message names its
 * index), LP_ENOMEM, LP_ECUDA. */
lp_status lp_batch_create(int32_t count, const lp_graph_desc *graphs, uint32_t flags,
                          void *cuda_stream, lp_batch **out);

/* Free a batch (NULL is a no-op). */
lp_status lp_batch_destroy(lp_batch *b);

/* Run RAK on every graph of the batch with the same parameters
 * (init_labels must be NULL).  per_graph[i] receives graph i's outcome
 * (array of `count` results, may be NULL).
 * Errors: as lp_rak_run. */
lp_status lp_batch_run(lp_batch *b, const lp_rak_params *p, lp_rak_result *per_graph);

/* ---------------------------------------------------------------------------
 * Bucket autotuning (no counterpart in the paper, which runs on a CPU).
 * Vertices are sorted into degree buckets, each swept by its own kernel
 * (several short rows per warp; one warp per row; one 128-, 256- or 512-thread
 * CTA per row; segments for the longest rows).  The autotuner times `sweeps`
 * iterations (tolerance 0, from unique labels, with p's mode / waves / tie
 * rule / seed) for each of 16 choices of the buckets' largest degrees within
 * the kernels' capacities (small <= 32, warp <= 128, cta <= 512, cta2 <= 1024)
 * and keeps the fastest.  Results of later runs do not depend on the choice.
 * Labels are left in an unspecified state; the next run starts afresh.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t small_max;   /* chosen largest degree of the small bucket */
    int32_t warp_max;    /* ... of the warp bucket */
    int32_t cta_max;     /* ... of the 128-thread CTA bucket */
    int32_t cta2_max;    /* ... of the 256-thread CTA bucket */
    int32_t candidates;  /* choices timed */
    float default_ms;    /* timed iterations with the default bounds (32/128/512/1024) */
    float best_ms;       /* timed iterations with the chosen bounds */
} lp_tune_result;

/* Autotune a batch's buckets (p->init_labels must be NULL; 1 <= sweeps <= 100).
 * Errors: LP_EINVAL on NULL arguments or a bad parameter; LP_ENOMEM; LP_ECUDA. */
lp_status lp_batch_autotune(lp_batch *b, const lp_rak_params *p, int32_t sweeps,
                            lp_tune_result *out);

/* Autotune a single graph's buckets (p->init_labels is ignored).
 * Errors: as lp_batch_autotune. */
lp_status lp_graph_autotune(lp_graph *g, const lp_rak_params *p, int32_t sweeps,
                            lp_tune_result *out);

/* Set the buckets' largest degrees directly (max_degree[4]: small, warp,
 * cta, cta2; non-decreasing, >= 1, at most 32 / 128 / 512 / 1024), e.g. an
 * autotuning result from a similar graph.
 * Errors: LP_EINVAL on NULL or out-of-range bounds; LP_ENOMEM; LP_ECUDA. */
lp_status lp_graph_set_buckets(lp_graph *g, const int32_t *max_degree);
lp_status lp_batch_set_buckets(lp_batch *b, const int32_t *max_degree);

/* Labels of graph `index` after the last lp_batch_run (n_index int32).
 * Errors: LP_EINVAL on NULL or index out of range; LP_ECUDA. */
lp_status lp_batch_labels_get(lp_batch *b, int32_t index, int32_t *dst, int32_t dst_on_device);

/* Modularity of graph `index` under its current labels (see lp_modularity).
 * Errors: LP_EINVAL; LP_ENOMEM; LP_ECUDA. */
lp_status lp_batch_modularity(lp_batch *b, int32_t index, double *q);

/* ---------------------------------------------------------------------------
 * Serving: a request server with continuous batching.
 * Each request is one graph run with the server's parameters.  An admission
 * thread admits queued requests while fewer than max_active requests are on
 * the device and their estimated footprints (about 40 n + 88 m bytes each)
 * fit the HBM budget still free.  The requests of at most cohort_max_entries
 * entries it finds queued together, up to max_cohort of them, form one
 * cohort; a larger request forms a cohort of its own.  A lone request is
 * ingested as a graph, several as one batch arena (lp_batch_create), on one
 * of the server's streams, by one of `admitters` threads, so that the
 * ingest of several cohorts overlaps.  A worker thread advances every cohort one RAK iteration
 * (Sec. 3.2) at a time, interleaved with the other cohorts; an iteration of
 * a cohort is one launch per degree bucket for all of its graphs, and graphs
 * that have converged are left out of its later iterations and give their
 * active slots back (their memory stays counted until the cohort retires).
 * When a cohort's last graph has finished, its requests are retired
 * (modularity, labels).  A request's result is the same as
 * that of lp_rak_run on its graph alone.  If a cohort's batch cannot be
 * ingested (an invalid graph), its requests are ingested one by one, so that
 * only the invalid ones fail.
 * ------------------------------------------------------------------------- */
typedef struct lp_server lp_server;

typedef struct {
    int64_t hbm_budget; /* device bytes admitted requests may hold together (default 8 GiB) */
    int32_t max_active; /* requests on the device at once (default 64) */
    int32_t streams;    /* CUDA streams the cohorts are spread over, 1..64 (default 8) */
    int32_t max_cohort; /* requests ingested and iterated together, >= 1 (default 16;
                           1 = every request on its own) */
    int32_t admitters;  /* threads that ingest admitted requests, 1..16 (default 2) */
    int64_t cohort_max_entries; /* a graph with more CSR entries is admitted on its own
                                   (default 2^18: launch-bound small graphs gain from
                                   sharing launches, larger ones keep the GPU busy alone) */
} lp_server_config;

typedef struct {
    int64_t request_id;
    int32_t status;     /* LP_OK, or the error that ended this request */
    int32_t iterations;
    int32_t converged;
    int32_t pad;
    double modularity;
    double queued_ms;   /* submit -> admitted */
    double latency_ms;  /* submit -> result ready (labels copied) */
} lp_serve_result;

/* Fill *cfg with the defaults.  Errors: LP_EINVAL on NULL. */
lp_status lp_server_config_default(lp_server_config *cfg);

/* Start a server on the current device with parameters *p (init_labels must
 * be NULL).  Errors: LP_EINVAL for bad arguments; LP_ENOMEM; LP_ECUDA. */
lp_status lp_server_create(const lp_server_config *cfg, const lp_rak_params *p,
                           lp_server **out);

/* Queue one request.  offsets/indices/weights are a HOST CSR as in
 * lp_graph_create (weights may be NULL); they are not copied at submit and
 * must stay valid and unchanged until the request's result has been polled.
 * labels_out (host, n int32, may be NULL) receives the final labels before the
 * result is posted.  Thread-safe.
 * Errors: LP_EINVAL for bad arguments; LP_ENOMEM if the request alone exceeds
 * the budget.  A CSR that fails validation is reported in its result. */
lp_status lp_server_submit(lp_server *s, int64_t request_id, int32_t n, int64_t m,
                           const int32_t *offsets, const int32_t *indices,
                           const int32_t *weights, int32_t *labels_out);

/* Move up to `capacity` finished results to out (in completion order);
 * *count receives how many.  Waits up to wait_ms for the first one.
 * Returns LP_ENOTREADY when none was available.  Thread-safe. */
lp_status lp_server_poll(lp_server *s, lp_serve_result *out, int32_t capacity, int32_t *count,
                         int32_t wait_ms);

/* Cohorts formed so far, requests that ran in a cohort of two or more (one
 * batch arena), and the largest cohort.  Thread-safe.
 * Errors: LP_EINVAL on NULL. */
lp_status lp_server_stats(lp_server *s, int64_t *cohorts, int64_t *batched, int64_t *largest);

/* Block until every submitted request has a result.  Errors: LP_EINVAL on NULL. */
lp_status lp_server_drain(lp_server *s);

/* Finish every submitted request, stop the worker and free the server
 * (NULL is a no-op).  Unpolled results are discarded. */
lp_status lp_server_destroy(lp_server *s);

/* ---------------------------------------------------------------------------
 * COPRA: community overlap propagation (Sec. 3.3)
 * ------------------------------------------------------------------------- */

/* COPRA parameters. */
typedef struct {
    int32_t max_labels; /* pairs a vertex keeps at most, 1 .. 64 (the paper tries 1-32) */
    double tolerance;   /* stop once at most tolerance * n vertices changed their best
                           label; [0, 1] (the paper suggests 0.01) */
    int32_t max_iter;   /* >= 1 */
    int32_t mode;       /* LP_SYNC or LP_ASYNC (waves as in lp_rak_params) */
    int32_t waves;      /* >= 1 in LP_ASYNC */
    int32_t strict;     /* tie rule for the best label, as in lp_rak_params */
    uint64_t seed;      /* non-strict tie key */
} lp_copra_params;

/* max_labels 4, tolerance 0.01, max_iter 20, LP_ASYNC with 31 waves, strict,
 * seed 0.  Errors: LP_EINVAL on NULL. */
lp_status lp_copra_params_default(lp_copra_params *p);

/* Run COPRA on a graph (Sec. 3.3).  Every vertex holds at most max_labels
 * (label, belonging) pairs, belongings in units of 2^-16 that sum to exactly
 * 2^16, stored by decreasing belonging (equal ones by first appearance), the
 * first pair being the vertex's best label; it starts as {(v, 2^16)}.  In an
 * iteration v sums T(l) = sum of w * b over its row's entries (u, w) and the
 * pairs (l, b) of u's set (its own labels are not added), keeps the labels
 * with max_labels * T(l) >= W * 2^16 (W: the row's summed weight), else the
 * best label alone (largest T; ties by the strict rule on first appearance,
 * or the non-strict tie key of iteration t), and stores the kept T divided
 * by their sum in fixed point (floor; the remainder to the best kept).  A
 * vertex without edges is its own community.  The run stops once at most
 * tolerance * n best labels changed, or after max_iter iterations.  The
 * graph's labels (lp_labels_get, lp_modularity) become the best labels; out
 * as for lp_rak_run, lp_rak_history gives the changed counts.
 * Errors: LP_EINVAL for NULL arguments, parameters out of range, or a row too
 * long for max_labels (its table would exceed 2^28 slots); LP_ENOMEM; LP_ECUDA. */
lp_status lp_copra_run(lp_graph *g, const lp_copra_params *p, lp_rak_result *out);

/* The sets of the last COPRA run: n x max_labels labels and belongings
 * (row-major, belonging 0 after a set's last pair; host or device by
 * dst_on_device).  Errors: LP_EINVAL (NULL, or no COPRA run yet); LP_ECUDA. */
lp_status lp_copra_sets_get(lp_graph *g, int32_t *labels, uint32_t *belongings,
                            int32_t dst_on_device);

/* ---------------------------------------------------------------------------
 * SLPA: speaker-listener label propagation (Sec. 3.4)
 * ------------------------------------------------------------------------- */

/* SLPA parameters. */
typedef struct {
    int32_t memory_size; /* labels each vertex remembers, slot 0 = the vertex itself;
                            1 .. 64 (at most memory_size - 1 iterations run) */
    double tolerance;    /* stop once at most tolerance * n vertices stored a label
                            that differs from their previous slot; [0, 1] */
    int32_t strict;      /* 1: the listener keeps the first of its heaviest spoken
                            labels (row order), 0: the one with the smallest tie key */
    uint64_t seed;       /* drives the speakers' slot draws and the non-strict key */
} lp_slpa_params;

/* memory_size 20, tolerance 0.05, strict 1, seed 0.  Errors: LP_EINVAL on NULL. */
lp_status lp_slpa_params_default(lp_slpa_params *p);

/* Run SLPA on a graph (Sec. 3.4): every vertex remembers its own id; in
 * iteration t = 1, 2, ... each neighbour u of a listener v speaks one label of
 * the slots 0 .. t-1 its memory held before the iteration, the slot drawn as
 * floor(hi32(h) * t / 2^32) from h = the counter-based SplitMix64 draw of
 * (seed ^ 0x5350454B, t, v, position of the entry in v's row) nested as in the
 * non-strict tie key; v sums the spoken labels' edge weights and stores the
 * heaviest in slot t (ties as in lp_rak_params with iteration index t).  A
 * vertex without edges repeats its previous slot.  Afterwards the graph's
 * labels (lp_labels_get, lp_modularity) are the communities: the label a
 * vertex's memory holds most often, the one stored first on equal counts.
 * out: iterations run, converged, the last iteration's changed count and the
 * device time; lp_rak_history gives the changed counts.  The memory
 * (memory_size x n int32) stays allocated with the graph.
 * Errors: LP_EINVAL for NULL arguments or parameters out of range; LP_ENOMEM;
 * LP_ECUDA. */
lp_status lp_slpa_run(lp_graph *g, const lp_slpa_params *p, lp_rak_result *out);

/* Copy memory slots 0 .. slots-1 of the last SLPA run to dst (slots x n int32,
 * slot t of vertex v at dst[t * n + v]; host or device, by dst_on_device);
 * slots may be at most the iterations run + 1.  Errors: LP_EINVAL; LP_ECUDA. */
lp_status lp_slpa_memory_get(lp_graph *g, int32_t *dst, int32_t slots, int32_t dst_on_device);

/* ---------------------------------------------------------------------------
 * One sweep without any allocation
 * ------------------------------------------------------------------------- */

/* One synchronous RAK sweep that allocates no memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device
 * memory at run time because their GPU memory is already fully reserved by
 * another allocator (a framework's caching allocator, or a pool sized once
 * under a fixed budget).  Every other entry point allocates; this one calls no
 * cudaMalloc, cudaFree or allocating library routine.
 *   n, m, offsets, indices, weights  a CSR as in lp_graph_create, all DEVICE
 *             pointers (weights may be NULL); it is validated like there and
 *             every row may hold at most 4096 entries (else LP_EINVAL).
 *   labels_in   n device labels in [0, n), read only.
 *   labels_out  n device labels, written; must differ from labels_in.
 *   strict, seed, iteration  tie rule, non-strict seed and the iteration
 *             index t of the non-strict key (see lp_rak_params).
 *   changed   host pointer, receives the number of vertices whose label changed.
 *   cuda_stream  stream for the work (NULL = legacy default stream); the call
 *             returns after the sweep has finished.
 * labels_out equals the labels after one iteration of lp_rak_run in LP_SYNC
 * mode started from labels_in with iter_offset = iteration.
 * Scratch: a file-scope device array of about 12.6 MB, held on every GPU that
 * loads the library until the process exits (the changed counter, the
 * validation status and per-CTA overflow tables).  The first call on a device
 * sets it up (looks up its device address, clears it) and synchronizes the
 * stream; make that first call before any stream capture.  All calls share the
 * array, so calls that overlap on the GPU (other threads, other streams) race
 * and their results are undefined; serialize them.
 * Errors: LP_EINVAL for NULL pointers, sizes out of range, an invalid CSR, a
 * row longer than 4096, labels outside [0, n), or labels_in == labels_out;
 * LP_ECUDA. */
lp_status lp_rak_sweep_noalloc(int32_t n, int64_t m, const int32_t *offsets,
                               const int32_t *indices, const int32_t *weights,
                               const int32_t *labels_in, int32_t *labels_out, int32_t strict,
                               uint64_t seed, int32_t iteration, int64_t *changed,
                               void *cuda_stream);

/* ---------------------------------------------------------------------------
 * Diagnostics
 * ------------------------------------------------------------------------- */

/* Device time of sweep launches, per kernel.  While profiling is enabled,
 * every sweep launch is bracketed by two CUDA events on the graph's stream
 * (a small overhead); the statistics accumulate across runs and graphs until
 * lp_profile_reset. */
typedef struct {
    char name[32];    /* "sweep_small", "sweep_warp", "sweep_cta", "sweep_cta2", "sweep_hub" */
    int64_t launches; /* profiled launches */
    double total_ms;  /* summed event time */
    double vertices;  /* vertices scheduled (summed over launches) */
    double entries;   /* CSR entries scheduled (summed over launches) */
    double bytes;     /* algorithmic HBM bytes: 12 per vertex (row pointer, own
                         label read, label write) + 4 per entry (column index)
                         + 4 per entry for weighted graphs */
} lp_kernel_stat;

/* Turn per-kernel profiling on (1) or off (0).  Always LP_OK. */
lp_status lp_profile_enable(int32_t on);

/* Clear the accumulated statistics.  Always LP_OK. */
lp_status lp_profile_reset(void);

/* Copy up to `capacity` kernel statistics to out; *count receives how many
 * kernels exist (5, one per degree bucket).  Errors: LP_EINVAL on NULL count,
 * or NULL out with capacity > 0. */
lp_status lp_profile_read(lp_kernel_stat *out, int32_t capacity, int32_t *count);

/* Measurement helper (no counterpart in the paper): the time of one pass that
 * streams the first m / 4 16-byte blocks of indices and weights (mode 0), or
 * also gathers labels[index] of every entry (mode 1), the data movement of a
 * sweep without its per-row work.  indices, weights (NULL = unit), labels
 * (n entries): device pointers, indices and weights 16-byte aligned, every
 * index in [0, n) (checked first, LP_EINVAL otherwise).  sink: two device
 * words, overwritten.  Runs 3 warm-up and `repeats` timed passes on
 * cuda_stream; *ms_per_pass receives their mean (CUDA events).
 * Errors: LP_EINVAL; LP_ECUDA. */
lp_status lp_probe_gather(int32_t n, int64_t m, const int32_t *indices, const int32_t *weights,
                          const int32_t *labels, int32_t mode, int32_t repeats, unsigned *sink,
                          float *ms_per_pass, void *cuda_stream);

/* Split every community of the graph's current labelling into its connected
 * components, in place: two vertices keep one label only if a path of edges
 * whose two ends both carry that label joins them.  The paper does not
 * post-process its communities and names this split as the step it leaves
 * out (end of Sec. 3.4).  Each component takes the id of its smallest vertex
 * as its label, so the result is unique; *communities (may be NULL) receives
 * the number of components, isolated vertices included.  Runs on the graph's
 * stream and synchronises it.  Single graphs only.
 * Errors: LP_EINVAL on NULL g, LP_ENOMEM, LP_ECUDA. */
lp_status lp_split_communities(lp_graph *g, int64_t *communities);

/* Self-test of the time limit on the grid barrier that the all-waves sweep
 * (asynchronous runs of 8 or more waves over rows of at most 32 entries)
 * waits at: four CTAs of one cooperative launch wait for a fifth that never
 * arrives, give up after 4096 polls and record the timeout.  *timed_out = 1
 * when they did; the CUDA context stays usable.  Synchronises the device.
 * Errors: LP_EINVAL on NULL, LP_ENOMEM, LP_ECUDA. */
lp_status lp_selftest_barrier_timeout(int32_t *timed_out);

/* Message of the last failed call on this thread ("" if none). */
const char *lp_last_error(void);

/* Number of kernels this library has launched in this process. */
int64_t lp_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* LP_H */
