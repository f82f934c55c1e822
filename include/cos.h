/*
 * cos.h -- C ABI of the GB300 combinatorial-summation (CoS) graph evaluator.
 *
 * The method (Sec. II.B, Fig. 1): a leveled directed graph whose top node holds
 * 1; every edge multiplies the value of its origin node by a propagator and
 * adds the product to its destination node; every node is the sum over its
 * in-edges; the last node holds the sum over all root-to-sink paths, one path
 * per Feynman diagram.  The graph is built once and evaluated for many Monte
 * Carlo samples of the vertex times (Sec. II.B last paragraph, Sec. IV).
 *
 * Conventions shared by every entry point
 *   - Levels l = 0..L-1.  Level l owns the contiguous global node ids
 *     [off_l, off_l + W_l), off_0 = 0.  W_0 = W_{L-1} = 1: node 0 is the root,
 *     node N-1 the sink (N = sum of W_l).
 *   - Edges are the flattened per-level lists of Fig. 3: int32 rows
 *     (src, dst, kind, i, j), level-major (level_edge_count[l] rows for level l,
 *     in increasing l).  Bit 30 of `kind` marks an edge that closes a fermion
 *     loop: its factor is multiplied by -1 (Sec. II.C, "Numerical stability");
 *     bits 0..29 hold the kind.  Every edge into level l has src in level l-1 and dst in
 *     level l.  Duplicate (src, dst) pairs are separate edges.
 *   - Edge factor for sample s: +-G_kind(t_{s,i} - t_{s,j}) with the free-fermion
 *     propagator G_k(tau) = -exp(-eps_k tau)/(1+exp(-beta eps_k)) for tau >= 0
 *     and G_k(tau) = -G_k(tau+beta) for tau < 0 (tau = 0 takes the first branch;
 *     the comparison is made on the double-precision times), unless
 *     cos_set_propagator_table gave the handle tables of G_k instead.
 *   - Device memory: every buffer the library allocates belongs to the graph
 *     handle and is freed by cos_destroy.  Output buffers passed in are owned by
 *     the caller.  All device work runs on the CUDA device that was current when
 *     the graph was created, on the stream passed in (NULL = legacy default
 *     stream).  One graph handle must be used by one stream at a time.
 *   - Every function returns COS_OK (0) or a negative cos_status.  On error,
 *     cos_last_error() returns a thread-local message; nothing aborts the
 *     process and no call leaves the CUDA context unusable.
 */
#ifndef COS_H_
#define COS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cos_graph* cos_graph_t;

enum cos_status {
    COS_OK = 0,
    COS_ERR_INVALID = -1,   /* bad argument or malformed graph; nothing was created or changed */
    COS_ERR_OOM = -2,       /* a device or host allocation failed */
    COS_ERR_CUDA = -3,      /* a CUDA runtime call failed (message in cos_last_error) */
    COS_ERR_TIMEOUT = -4,   /* a bounded wait inside a kernel (grid barrier, work-queue dependency,
                               bulk-copy barrier) gave up; results are invalid, the context is usable */
    COS_ERR_OVERFLOW = -5,  /* count mode: the exact path count exceeds 2^63-1 (results wrap mod 2^64) */
    COS_ERR_STATE = -6,     /* call out of order, e.g. cos_evaluate before cos_set_samples */
    COS_ERR_BUSY = -7       /* resident server: the request is still running (poll), or no request
                               slot or queue space is free right now (submit; retry later) */
};

enum cos_mode {
    COS_MODE_FP64 = 0,        /* propagators, products and sums in IEEE double */
    COS_MODE_FP32_MIXED = 1,  /* propagators (formed in double, rounded once) and per-level products
                                 in float; sink node and cross-sample sums in double, compensated */
    COS_MODE_COUNT_I64 = 2,   /* unit edge weights, int64 sums modulo 2^64: the number of paths */
    COS_EVAL_ABS = 16         /* flag, with modes 0 and 1: the same walk also accumulates
                                 A(s) = sum over paths of |path value| (every factor replaced by
                                 its absolute value), the scale against which the accuracy of R(s)
                                 is stated.  A's node values and products are float (about 1e-6
                                 relative: a scale, not a result), its sink and sample sums double.
                                 Results double: per-sample outputs hold 2*S values (R(s) for s < S,
                                 then A(s)), means two (mean R, mean A).  Wide layout only. */
};

enum cos_t_flags {
    COS_T_DEVICE_DS = 0,      /* t is a device pointer, layout [D][S] (sample index fastest) */
    COS_T_HOST = 1,           /* t is a host pointer (page-locked memory gives an asynchronous copy) */
    COS_T_SAMPLE_MAJOR = 2,   /* layout [S][D] (time-variable index fastest) */
    COS_T_BORROW = 4          /* device [D][t_ld] buffer, t_ld = S rounded up to 128, used in place
                                 without a copy: it must stay valid and unchanged until the last
                                 evaluation of these samples has finished; padding must be finite */
};

/*
 * Graph ingest (Sec. II.C "Graph flattening", Fig. 3).  Validates the levels
 * and edges, buckets them per level, stable-sorts each level by destination
 * into CSR form (the in-edges of one node stay in input order), numbers the
 * distinct (kind, i, j) triples as propagator slots, counts root-to-sink paths
 * exactly on the host (128-bit, for the count-mode overflow flag), and copies
 * the result to the current device.
 *   num_levels         L >= 2
 *   level_width[L]     host, W_l >= 1, W_0 = W_{L-1} = 1, N = sum W_l < 2^31
 *   level_edge_count[L] host, [0] == 0, [l] >= 0, E = sum < 2^31
 *   edges[E][5]        host, int32 rows (src, dst, kind, i, j) as above
 *   num_kinds K >= 1, 1 <= num_times D <= 192 (kind < K, i, j < D)
 *   out                receives the handle; untouched on error
 * The caller keeps ownership of its arrays; they are not referenced afterwards.
 * Errors: COS_ERR_INVALID (any violation, message names it), COS_ERR_OOM, COS_ERR_CUDA.
 */
int cos_create_graph(int32_t num_levels, const int64_t* level_width, const int64_t* level_edge_count,
                     const int32_t* edges, int32_t num_kinds, int32_t num_times, cos_graph_t* out);

/*
 * A second handle on the structure of `src` (levels, CSR, propagator slots stay
 * on the device once, shared): the new handle has its own samples, workspace and
 * results, so several sample sets of one resident graph can be evaluated
 * concurrently (e.g. one per in-flight request).  The structure is freed with the
 * last handle that uses it; handles may be destroyed in any order.
 * Errors: COS_ERR_INVALID, COS_ERR_OOM, COS_ERR_CUDA.
 */
int cos_graph_share(cos_graph_t src, cos_graph_t* out);

/*
 * Attach a batch of Monte Carlo samples (Sec. II.C "Distributing the task on a
 * grid of blocks": one evaluation per set of internal variables).
 *   num_samples S >= 0
 *   t        S x D doubles, layout and location given by t_flags (cos_t_flags);
 *            values are the imaginary times, expected in [0, beta)
 *   eps[K]   host doubles, the per-kind energies
 *   beta     inverse temperature (> 0)
 *   stream   cudaStream_t (as void*) on which the copy is enqueued
 * Grows the graph's device workspace if needed; a tile_samples tuning fixes the
 * workspace to that many samples (set it before the first cos_set_samples).
 * (Device memory is otherwise allocated by cos_create_graph, cos_graph_share,
 * cos_set_propagator_table, cos_mc_create, and on first use of the work-queue
 * schedule or of an internal result buffer; cos_evaluate_static never allocates.)
 * The copy is asynchronous: a host t must stay valid until the stream reaches
 * this point.
 * Errors: COS_ERR_INVALID, COS_ERR_OOM, COS_ERR_CUDA.
 */
int cos_set_samples(cos_graph_t g, int64_t num_samples, const double* t, int32_t t_flags,
                    const double* eps, double beta, void* stream);

/*
 * Attach S Monte Carlo samples drawn on the device (the integration over vertex
 * times by stochastic sampling, Sec. II.B; device-side sampling, Sec. IV): for
 * sample n = first_sample + s and time i, t[s][i] = beta * u with u in [0, 1) taken
 * from a counter-based generator -- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw,
 * SC'11) with counter (n mod 2^32, n >> 32, i / 2, 0) and key (seed mod 2^32,
 * seed >> 32), u = ((w1 << 32 | w0) >> 11) * 2^-53 for even i and the same from
 * (w3, w2) for odd i.  Successive batches of one Monte Carlo run continue the
 * stream by advancing first_sample; no host copy of times is needed.
 * Errors: as cos_set_samples.
 */
int cos_set_samples_uniform(cos_graph_t g, int64_t num_samples, uint64_t seed, int64_t first_sample,
                            const double* eps, double beta, void* stream);

/*
 * Copy the attached times to dst ([D][S] doubles, sample index fastest; device or
 * host memory), asynchronously on stream -- e.g. to keep the samples a Monte Carlo
 * batch was evaluated on.  Errors: COS_ERR_STATE without samples.
 */
int cos_copy_times(cos_graph_t g, double* dst, void* stream);

/*
 * Evaluate the path sum of every attached sample (Fig. 1; Sec. II.C): one
 * persistent kernel computes, tile of samples by tile, the propagator table,
 * walks the levels in order, writes the sink value per sample, and finally
 * reduces the samples -- either level-synchronous (cooperative launch, a
 * grid-wide barrier between levels) or from a work queue (see cos_tuning.schedule).
 * The level-synchronous schedule allocates nothing when per_sample_out is given
 * (without it, the first evaluation of a larger sample set allocates an internal
 * result buffer) and may then be captured in a CUDA graph when mean_out is NULL;
 * the work-queue schedule plans its task list on every call and uploads it when it
 * changed (a host wait for the previous upload's copy to run precedes a new
 * upload; buffers are allocated on first use), so it is not meant for capture.
 *   mode            cos_mode, optionally | COS_EVAL_ABS (modes 0 and 1)
 *   per_sample_out  device pointer or NULL: double[S] (FP64, FP32_MIXED) or
 *                   int64[S] (COUNT_I64), index = sample index; with COS_EVAL_ABS
 *                   double[2*S]: R(s) at s, A(s) at S + s
 *   mean_out        host pointer or NULL.  If non-NULL the call waits for the
 *                   stream and stores the mean over samples (Neumaier-compensated
 *                   double; in count mode the mean of the counts), and reports
 *                   kernel-side errors; with COS_EVAL_ABS mean_out[0] = mean R and
 *                   mean_out[1] = mean A (two doubles).  If NULL the call returns
 *                   at once; use cos_get_result to wait and collect.
 * Errors: COS_ERR_STATE (no samples attached), COS_ERR_INVALID (mode),
 *         COS_ERR_CUDA, COS_ERR_TIMEOUT, COS_ERR_OVERFLOW (count mode, exact
 *         count > 2^63-1; the wrapped results are still written).
 */
int cos_evaluate(cos_graph_t g, int32_t mode, void* per_sample_out, double* mean_out, void* stream);

/*
 * As cos_evaluate, with every edge factor replaced by its absolute value (the
 * fermion-loop sign ignored): per_sample_out receives A(s), the sum over paths of
 * |path value| -- the scale against which the accuracy of R(s) is stated (a
 * result has relative error eps when |R_computed - R_exact| <= eps * A) -- and
 * mean_out its mean.  Modes 0 and 1 only (COS_ERR_INVALID otherwise).
 */
int cos_evaluate_abs(cos_graph_t g, int32_t mode, void* per_sample_out, double* mean_out, void* stream);

/*
 * Wait for the last cos_evaluate on this graph (stream = the one it ran on) and
 * return its status; if mean_out is non-NULL store its mean there (two doubles,
 * mean R and mean A, when that evaluation had COS_EVAL_ABS).
 */
int cos_get_result(cos_graph_t g, double* mean_out, void* stream);

/*
 * User-tabulated propagators (Fig. 1 caption: the edge factor is a general
 * Green's function G; Sec. II.C "Numerical stability": every edge applies its
 * own propagator).  Replaces the free-fermion formula of every kind k of g by
 * numbers: table is host memory [K][2][T+1] doubles (copied; the caller keeps
 * ownership); half 0 holds G_k at tau = m*h, m = 0..T, h = tau_max/T, and is used
 * for tau = t_i - t_j >= 0; half 1 holds G_k at tau = -tau_max + m*h and is used
 * for tau < 0 (two halves keep the jump at tau = 0).  Between grid nodes the value
 * is the linear interpolation of its neighbours, computed in double and rounded
 * once to the mode's propagator type; outside [-tau_max, tau_max] the end value.
 * The fermion-loop sign (kind bit 30) still applies.  T = 0 (table and tau_max
 * ignored) returns to the formula.  1 <= T <= 2^24, tau_max finite and > 0,
 * every entry finite, else COS_ERR_INVALID and nothing changes.  The tables
 * belong to the handle: cos_graph_share copies them into the new handle.
 * Cost: about 7 FP64 operations per propagator slot and sample instead of one
 * multiplication (no exponentials).
 */
int cos_set_propagator_table(cos_graph_t g, int32_t T, const double* table, double tau_max);

/*
 * Metropolis walkers over the vertex times (Sec. II.B: the sum over diagrams is
 * integrated over the times by Monte Carlo sampling; Sec. II.C "Distributing the
 * task": many Markov-chain walkers on one GPU; Sec. III: proposal and acceptance
 * in device code).  Every sample attached to g is a walker and its times are the
 * starting configuration; the walkers' state IS the graph's time buffer (with
 * COS_T_BORROW, the caller's buffer), read back with cos_copy_times.
 *   cos_mc_create  mode 0 (FP64) or 1 (FP32 mixed); evaluates R at the start
 *                  (COS_ERR_STATE without samples, COS_ERR_INVALID for count mode)
 *   cos_mc_run     num_steps steps, all on `stream`: walker s at step n draws
 *                  Philox-4x32-10 words w0..w3 (counter (s mod 2^32, s >> 32,
 *                  n mod 2^32, 2^31 | n >> 32), key (seed mod 2^32, seed >> 32)),
 *                  replaces time i = (w0*D) >> 32 by beta*(((w2<<32|w1)>>11)*2^-53),
 *                  evaluates every walker (cos_evaluate, the graph's tuning), keeps
 *                  the move iff (w3 + 1/2)*2^-32 * |R| < |R'|, and tallies the sign
 *                  of its current R
 *   cos_mc_stats   out[4] = steps, accepted moves, positive and negative tallies
 *                  (64-bit, exact); synchronizes `stream` and returns the status of
 *                  the last evaluation.  (pos - neg)/(pos + neg) estimates the ratio
 *                  of the integrals of R and |R| over [0, beta)^D.
 *   cos_mc_values  copies the walkers' current R (double [S], host or device)
 * The walkers must not outlive g, and g's samples must not be replaced while they
 * run (COS_ERR_STATE).  The paper has the scheme, not this interface.
 */
typedef struct cos_mc* cos_mc_t;
int cos_mc_create(cos_graph_t g, int32_t mode, uint64_t seed, void* stream, cos_mc_t* out);
int cos_mc_run(cos_mc_t m, int32_t num_steps, void* stream);
int cos_mc_stats(cos_mc_t m, int64_t* out, void* stream);
int cos_mc_values(cos_mc_t m, double* per_walker_out, void* stream);
int cos_mc_destroy(cos_mc_t m);

/*
 * Graph facts, written to info[0..n) in this order (n <= 10):
 *   0 L, 1 N, 2 E, 3 number of propagator slots P, 4 widest level W_max,
 *   5 path count mod 2^64 (from ingest), 6 path-count overflow flag,
 *   7 K, 8 D, 9 device ordinal
 */
int cos_graph_info(cos_graph_t g, int64_t* info, int32_t n);

/*
 * Launch shape used by cos_evaluate.  Fields <= 0 mean "automatic".
 *   samples_per_lane  1, 2 or 4 consecutive samples per thread (vector width)
 *   tile_samples      samples per tile (rounded up to 32 * samples_per_lane)
 *   rows_per_warp     consecutive destination rows one warp takes per work item (<= 31);
 *                     automatic: 31 with the work queue (16 in FP32 mixed mode when
 *                     every level has fewer than 65536 nodes), else 4 (FP64), 8 (FP32
 *                     mixed) or 16 (count)
 *   blocks_per_sm     persistent CTAs per SM (capped by occupancy)
 *   timeout_ms        limit of every bounded wait in the kernels (grid barrier,
 *                     work-queue dependency, bulk-copy barrier); default 10 s
 *   layout            1 = wide (a warp owns one row; chunks of 32*samples_per_lane
 *                     samples), 2 = grouped (a warp owns samples_per_lane rows, each
 *                     served by 32/samples_per_lane lanes; chunks of 32 samples),
 *                     3 = wide with a bulk-copy ring (one lane stages whole parent
 *                     and propagator runs in shared memory with cp.async.bulk on
 *                     mbarriers, 8 edges in flight per warp), 4 = wide with an
 *                     async-copy ring (every lane stages its own values of the parent
 *                     and propagator runs with cp.async, 6 edges in flight per warp
 *                     without registers)
 *   schedule          1 = level-synchronous: one cooperative kernel, every level of a
 *                     tile ends at a grid-wide barrier, work items assigned
 *                     statically; 2 = work queue (Sec. II.C, asynchronous evaluation
 *                     of levels): the persistent work-queue kernel of the batched
 *                     launch, items drawn from a ticket counter, each waiting only for
 *                     the previous phase of its own window of sample chunks.  The
 *                     chunks of each tile are cut into windows of window_chunks
 *                     chunks; every window is its own chain (propagators, levels
 *                     1..L-1, continuing into the same window of the next tile) and
 *                     the chains are issued in wavefront order, so about L windows
 *                     are in flight.  Results are bitwise the same either way.
 *                     Automatic: 2 in FP64 and FP32 mixed modes with at least 1e9
 *                     edge x samples or when the widest level has at least 65536
 *                     nodes, else 1.
 *                     Batched launches always use the
 *                     work queue, with windows when window_chunks > 0.
 *   window_chunks     chunks (of 32*samples_per_lane samples, 32 in the grouped
 *                     layout) per window of the work-queue schedule; automatic: a
 *                     quarter of a tile's chunks (four windows per tile)
 *   prefetch          wide layout: 1 = off; 2 = on levels whose parent slice per
 *                     chunk (previous level's width x chunk samples x value size)
 *                     exceeds 32 MB, i.e. does not stay in L2 (automatic); 3 = on
 *                     every level.  When on, each warp issues an L2 prefetch of the
 *                     next 4 edges' parent runs while it loads the current 4.
 *                     4 and 5: as 2 and 3, but every lane of a warp issues one bulk
 *                     L2 prefetch (cp.async.bulk.prefetch) of a whole parent run, for
 *                     the 32 edges of the next metadata window (and of the first).
 *                     6 and 7: as 2 and 3, prefetching the batch of 4 edges after the
 *                     next.
 */
typedef struct cos_tuning {
    int32_t samples_per_lane;
    int32_t tile_samples;
    int32_t rows_per_warp;
    int32_t blocks_per_sm;
    int32_t timeout_ms;
    int32_t layout;
    int32_t schedule;
    int32_t window_chunks;
    int32_t prefetch;
} cos_tuning;

int cos_set_tuning(cos_graph_t g, const cos_tuning* tuning);
/* Tuning cos_evaluate will use for `mode` with the current samples (automatic fields resolved). */
int cos_get_tuning(cos_graph_t g, int32_t mode, cos_tuning* tuning);
/*
 * Time launch shapes for `mode` on g's attached samples (both schedules, 8/16/31
 * rows per warp, two vector widths; fields already set > 0 stay fixed), keep the
 * fastest as g's tuning and, if best is non-NULL, store its resolved form there.
 * Runs 36 evaluations at most on `stream` (writing per_sample_out, which may be
 * NULL) and synchronizes; results are bitwise the same for every candidate.
 * The paper has no counterpart; cos_batch_autotune does the same for batches.
 */
int cos_autotune(cos_graph_t g, int32_t mode, void* per_sample_out, void* stream, cos_tuning* best);

/*
 * Batched evaluation of many graphs of uneven size and sample count in ONE
 * persistent launch (Sec. III "Acceleration" notes that small graphs leave most
 * of a thread block idle and suggests packing several small levels per block;
 * Sec. II.C "Windowing" suggests evaluating levels asynchronously).  Every graph's
 * work is cut into CTA-sized items (propagator factors and table per tile of
 * samples, each level per tile, the sample reduction); the per-graph phase chains
 * are interleaved into one task list that a persistent grid drains through a
 * ticket counter, each item waiting only for the previous phase of its own graph
 * (of its own window of sample chunks when window_chunks > 0).
 * The launch (counter reset + kernel) is captured into a CUDA graph on first use
 * and replayed by every later cos_batch_launch.
 *
 *   cos_batch_create  n distinct graph handles (each with samples attached, all on
 *                     one device), one mode for the batch (optionally | COS_EVAL_ABS:
 *                     then per-sample outputs hold 2*S doubles as in cos_evaluate),
 *                     per_sample_outs[n]
 *                     device pointers (entries may be NULL; NULL array = none).
 *                     The handles must outlive the batch.  Re-attaching samples to
 *                     a member, or changing its tuning or propagator tables, makes
 *                     the next cos_batch_launch plan again (and capture again): the
 *                     plan holds the member's buffers and sizes.
 *   cos_batch_reset   replace the members (same rules as create) keeping the device
 *                     buffers; the previous launch must have been collected.
 *   cos_batch_set_tuning  batch-wide overrides (fields > 0): samples_per_lane and
 *                     layout (one value for the launch), rows_per_warp,
 *                     tile_samples, blocks_per_sm, timeout_ms, window_chunks,
 *                     prefetch; other fields come from each graph.
 *   cos_batch_autotune  times every (samples_per_lane, rows_per_warp, layout)
 *                     candidate on the batch itself, keeps the fastest and returns
 *                     it in *best.
 *   cos_batch_launch  enqueue one evaluation of all graphs on `stream`.  The first
 *                     launch of a plan uploads it (stream-ordered) and runs the
 *                     kernel directly; the second captures counter reset + kernel
 *                     into a CUDA graph, which every later launch replays.
 *   cos_batch_results wait for `stream`; means[n] (host, may be NULL) receives each
 *                     graph's mean -- means[n][2] (mean R, mean A) for a batch whose
 *                     mode has COS_EVAL_ABS; errors as cos_evaluate (COS_ERR_TIMEOUT
 *                     if a dependency wait gave up).
 *   cos_evaluate_batch  modes[n]: a cos_mode per graph (optionally | COS_EVAL_ABS);
 *                     the graphs of each distinct mode form one batch (one persistent
 *                     launch each, all enqueued on `stream` before the first wait),
 *                     created, launched, collected and destroyed in this call.
 *                     per_sample_outs as cos_batch_create (NULL = none);
 *                     means[n][2] (host, may be NULL): [g][0] = mean R of graph g,
 *                     [g][1] = its mean A with COS_EVAL_ABS, else NaN.
 * Per-sample results are identical to cos_evaluate's for the same tuning.
 */
typedef struct cos_batch* cos_batch_t;
int cos_batch_create(int32_t n, const cos_graph_t* graphs, int32_t mode, void* const* per_sample_outs,
                     cos_batch_t* out);
int cos_batch_reset(cos_batch_t b, int32_t n, const cos_graph_t* graphs, void* const* per_sample_outs);
int cos_batch_set_tuning(cos_batch_t b, const cos_tuning* tuning);
int cos_batch_get_tuning(cos_batch_t b, cos_tuning* tuning);
int cos_batch_autotune(cos_batch_t b, void* stream, cos_tuning* best);
int cos_batch_launch(cos_batch_t b, void* stream);
int cos_batch_results(cos_batch_t b, double* means, void* stream);
int cos_batch_destroy(cos_batch_t b);
int cos_evaluate_batch(int32_t n, const cos_graph_t* graphs, const int32_t* modes, void* const* per_sample_outs,
                       double* means, void* stream);

/*
 * Phase trace (profiling aid; the paper reports only FLOPS).  cos_set_trace(g, n)
 * with n > 0 allocates room for n records and makes every later cos_evaluate on
 * g record, at each grid barrier, the %globaltimer value (ns) when CTA 0 passed
 * it and the phase id (0 = kernel start, 1 = coefficients, 2 = propagator table
 * of a tile (exponentials and products), 3+l = level l, 1000 = sample partial
 * sums).  n = 0 frees it.  cos_get_trace waits for the device, copies up to
 * `capacity` (time, phase) pairs of the last evaluate into out[2*capacity] and
 * stores how many were written in *count.
 */
int cos_set_trace(cos_graph_t g, int32_t capacity);
int cos_get_trace(cos_graph_t g, int64_t* out, int32_t capacity, int32_t* count);

/*
 * cos_evaluate_static -- evaluate an existing graph without allocating device memory.
 *
 * The paper has no counterpart.  This entry point is for callers that must not
 * call cudaMalloc or cudaFree while they evaluate: a host framework whose own
 * caching allocator owns the device memory budget (an allocation by this library
 * would fail or fragment its pool), and latency-bound serving loops, where
 * cudaMalloc and cudaFree can synchronise the device and stall other streams.
 * Such callers create the graph once at set-up time (cos_create_graph allocates)
 * and then call this function with their own device buffers for the times,
 * energies and results.
 *
 * Scratch memory.  The working memory of the evaluation -- the node-value slabs
 * and propagator table of one tile of samples, the per-kind coefficients, the
 * partial sums of the sample reduction, the grid-barrier counter, the error word
 * and the result -- lives in one file-scope __device__ array of
 * COS_STATIC_SCRATCH_BYTES (64 MiB) inside the library; every GPU that loads the
 * library holds it until the process exits.  The function calls no cudaMalloc,
 * cudaFree or other allocating routine.  The barrier counter and result are
 * cleared on every call; the rest keeps the last call's contents and is
 * overwritten before use.  Every call on a device shares the one array, so calls
 * whose execution overlaps on the GPU (different streams, or host threads) race
 * and give wrong results: serialise them.  Set-up: the first call on a device,
 * with that device current, looks up the array's device address
 * (cudaGetSymbolAddress, which may load the module); it is looked up again only
 * if the device's context changes.  Make that first call before any stream
 * capture begins.
 *
 * Errors from the kernel.  With mean_out == NULL the call returns right after the
 * launch.  A bounded wait that gives up inside the kernel (limit: the handle's
 * timeout_ms tuning, default 10 s) leaves a failure recorded in the array; the
 * next call that passes mean_out returns COS_ERR_TIMEOUT for it and clears it.
 * The results of every call from the failed one up to that reporting call are
 * then invalid.  A call with num_samples = 0 and mean_out non-NULL collects the
 * status cheaply.
 *
 * Limits.  The tile of samples is sized to fit the array; a graph whose working
 * set for 32 samples exceeds it (roughly 2 * W_max * w + P * w bytes
 * per sample, w = 8 in FP64 and count modes, 4 in FP32 mixed mode) is rejected
 * with COS_ERR_INVALID, as is a sample count whose partial sums do not fit.
 *
 *   g               graph from cos_create_graph; its device must be current
 *   mode            cos_mode
 *   num_samples     S >= 0
 *   t               device, layout [D][t_ld] (sample index fastest); t_ld >= S
 *                   rounded up to a multiple of 128; the padding columns are
 *                   read (must be finite) but do not affect any result
 *   eps             device, [K] doubles
 *   beta            inverse temperature (> 0)
 *   per_sample_out  device, double[S] (FP64, FP32_MIXED) or int64[S] (COUNT_I64);
 *                   required when S > 0
 *   mean_out        host pointer or NULL; non-NULL waits for the stream, stores
 *                   the mean over samples and reports kernel-side errors (above)
 *   stream          cudaStream_t as void*
 * Results equal those of cos_evaluate on the same samples (the per-sample sums
 * do not depend on the tile size).  Errors: as cos_evaluate, plus
 * COS_ERR_INVALID for the size limits above.
 */
#define COS_STATIC_SCRATCH_BYTES (64LL * 1024 * 1024)
int cos_evaluate_static(cos_graph_t g, int32_t mode, int64_t num_samples, const double* t, int64_t t_ld,
                        const double* eps, double beta, void* per_sample_out, double* mean_out, void* stream);

/*
 * Self test of the evaluator's double-precision exponentials: em[q] = e^{-x[q]},
 * ep[q] = e^{+x[q]} for device arrays of n doubles, |x| <= 708, computed exactly as
 * the propagator phase computes them (table-driven method, P. T. P. Tang, ACM TOMS
 * 15 (1989)).  g supplies the device and the 2^{j/64} table.  Asynchronous on stream.
 */
int cos_selftest_exp(cos_graph_t g, int64_t n, const double* x, double* em, double* ep, void* stream);

/*
 * Throughput of the fused multiply-add pipe of the current device, measured by a
 * probe kernel: *fma_per_second receives multiply-adds per second (precision 0:
 * double, 1: float) -- the denominator of the arithmetic roofline of the FP64
 * walk, whose every edge and sample is one double multiply-add (Fig. 1: the
 * parent's value times the propagator, added to the child).  Synchronous; takes a
 * few milliseconds; allocates and frees a small output buffer.
 * Errors: COS_ERR_INVALID, COS_ERR_CUDA.
 */
int cos_probe_fma_rate(int32_t precision, double* fma_per_second);

/*
 * Resident server (continuous batching at work-item granularity).  One persistent
 * kernel keeps running while requests arrive; a request is one evaluation of a
 * graph handle (Fig. 1; Sec. II.C) over counter-based uniform sample times drawn
 * on the device (the generator of cos_set_samples_uniform), cut into the same
 * work items as a batched launch.  The host feeds the tasks of all active requests
 * into a task queue in device memory round-robin (one task per request per round,
 * as the batched plan interleaves graphs), through host-to-device copies on a
 * stream of the server's own, keeping a bounded backlog ahead of the kernel: a
 * request admitted while the kernel runs joins the rotation within that backlog --
 * no launch boundary, and no kernel has to run to admit it.  Feeding happens inside
 * submit, poll, wait and stats, so a caller with requests in flight keeps calling
 * poll or wait.  CTAs that find no work for idle_ms leave; the next call relaunches
 * the kernel when work is pending.  Completion is reported through host-mapped
 * records that poll and wait read without synchronising a stream.
 *
 *   cos_server_create  mode (one per server); max_times = the largest D of the
 *                      graphs to be served (sizes shared memory); tuning (NULL or
 *                      fields > 0): samples_per_lane, rows_per_warp (default 31),
 *                      tile_samples, blocks_per_sm, timeout_ms (dependency waits,
 *                      default 10000), window_chunks, prefetch; layout must be 0 or
 *                      1 (wide).  max_requests (default 256) request slots;
 *                      queue_tasks (default 65536, rounded up to a power of two)
 *                      task entries (the backlog is min(queue_tasks/2, 16384));
 *                      idle_ms (default 50).  Allocates everything
 *                      it will use (nothing is allocated while serving).  The
 *                      server belongs to the device current at creation.
 *   cos_server_submit  evaluate handle g over num_samples samples numbered
 *                      first_sample.. of generator key `seed`; per-sample values go
 *                      to per_sample_out (device, max(num_samples,1) doubles, or
 *                      int64 in count mode; required).  The running kernel may write
 *                      them as soon as the request is submitted, unordered with the
 *                      caller's streams: work on other streams that uses that buffer
 *                      must be complete before submit.  g must have had a sample
 *                      set of at least num_samples attached in its own buffer
 *                      (cos_set_samples_uniform, or cos_set_samples without
 *                      COS_T_BORROW) so that eps, beta and the buffers exist; the
 *                      request overwrites the handle's times and sample count.  A
 *                      handle serves one request at a time (COS_ERR_STATE while
 *                      busy: use cos_graph_share for concurrent requests on one
 *                      graph).  *request_id receives the request number.
 *                      COS_ERR_BUSY: no free request slot (nothing changed;
 *                      collect results and retry).
 *   cos_server_poll    COS_OK with *mean_out (may be NULL) once the request is
 *                      complete (the request is then collected and its id becomes
 *                      invalid), COS_ERR_BUSY while it runs, or its error
 *                      (COS_ERR_TIMEOUT if a dependency wait gave up; then every
 *                      pending request fails and the server must be destroyed;
 *                      COS_ERR_OVERFLOW in count mode as cos_evaluate).
 *   cos_server_wait    poll until not busy or timeout_ms (< 0: no limit) passed
 *                      (then COS_ERR_TIMEOUT; the request stays pending).
 *   cos_server_stats   counters (below).
 *   cos_server_destroy finish every submitted request (unless the server failed),
 *                      stop the kernel, free everything.
 * One host thread per server.  Sample times of a request live in the handle's own
 * buffer until its next request; per_sample_out is written before completion is
 * reported.
 */
typedef struct cos_server* cos_server_t;
typedef struct cos_server_info {
    int64_t launches;         /* kernel launches so far (1 + relaunches after idle exits) */
    int64_t completed;        /* requests completed */
    int64_t in_flight;        /* requests submitted and not complete */
    int64_t queued_tasks;     /* task entries published and not yet complete (in order) */
    int64_t published_tasks;  /* tasks published since creation */
    int32_t running;          /* 1 while the kernel has CTAs resident */
    int32_t grid;             /* CTAs per launch */
    int32_t samples_per_lane;
    int32_t failed;           /* 0, or the cos_status every pending request fails with */
    int64_t stale_claims;     /* items claimed through a cursor value a whole queue behind (the
                                 slot already held a later task, whose item was taken instead) */
} cos_server_info;
int cos_server_create(int32_t mode, int32_t max_times, const cos_tuning* tuning, int32_t max_requests,
                      int64_t queue_tasks, int32_t idle_ms, cos_server_t* out);
int cos_server_submit(cos_server_t s, cos_graph_t g, int64_t num_samples, uint64_t seed, int64_t first_sample,
                      void* per_sample_out, int64_t* request_id);
int cos_server_poll(cos_server_t s, int64_t request_id, double* mean_out);
int cos_server_wait(cos_server_t s, int64_t request_id, int32_t timeout_ms, double* mean_out);
int cos_server_stats(cos_server_t s, cos_server_info* info);
int cos_server_destroy(cos_server_t s);

/* Free every device and host resource of the handle (NULL is accepted). */
int cos_destroy(cos_graph_t g);

/* Thread-local message describing the last non-OK return on this thread. */
const char* cos_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* COS_H_ */
