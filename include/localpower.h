/*
 * localpower.h -- C ABI of the GB300 LocalPower library.
 *
 * LocalPower (Li, Wang, Chen & Zhang, "Communication-Efficient Distributed SVD
 * via Local Power Iterations", ICML 2021) computes the top-k right singular
 * subspace of a row-partitioned matrix A = [A_1; ...; A_m] (Sec. 1, problem
 * statement; Alg. 1).  Here the m partitions are device-resident row blocks of
 * one GPU; a "communication round" of the paper is one on-device aggregation.
 *
 * Conventions shared by every call:
 *   - Matrices are row-major.  A partition A_i is s_i x d with row pitch d
 *     elements as given by the caller (the library repacks it internally).
 *   - Pointers are plain host or device pointers, as the lp_ptr_space argument
 *     says.  The library never keeps a caller pointer after a call returns.
 *   - Every call returns an lp_status.  No call aborts, throws or exits; after a
 *     non-OK status lp_last_error() describes the failure.  A failed call leaves
 *     the context usable unless the status is LP_ERR_CUDA (device context lost).
 *   - One context is used by one host thread at a time.  Distinct contexts may
 *     share a device.
 */
#ifndef LOCALPOWER_H
#define LOCALPOWER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LP_ABI_VERSION 1
#define LP_MAX_K 32

typedef enum lp_status {
    LP_OK = 0,
    LP_ERR_INVALID = 1,     /* bad argument; nothing was launched or allocated   */
    LP_ERR_STATE = 2,       /* call out of order (e.g. solve before load)        */
    LP_ERR_OOM = 3,         /* HBM budget or device memory exhausted             */
    LP_ERR_CUDA = 4,        /* a CUDA runtime call failed                        */
    LP_ERR_NUMERIC = 5,     /* Cholesky breakdown, non-finite data or iterate    */
    LP_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up                */
    LP_ERR_UNSUPPORTED = 7  /* valid request this build has no kernel for        */
} lp_status;

typedef enum lp_dtype {
    LP_F32 = 0,             /* IEEE binary32                                      */
    LP_BF16 = 1,            /* bfloat16 bit patterns (uint16)                     */
    LP_FP8_E4M3 = 2,        /* OCP FP8 E4M3 "FN" codes (uint8) x one FP32 scale per row */
    LP_F32_BF16X2 = 3       /* IEEE binary32 input, stored on the device as two bfloat16
                             * planes hi = RNE(a), lo = RNE(a - hi) (same 4 bytes per
                             * element) and multiplied on the tensor cores.  The stored
                             * matrix hi + lo differs from a by at most 2^-17 |a|. */
} lp_dtype;

/* The aligning family F of the unified update rule (App. B): F = {I} gives vanilla
 * averaging, F = diagonal +-1 matrices gives sign-fixing (eq. (4)), F = O_k gives
 * the orthogonal Procrustes transformation (eq. (3)). */
typedef enum lp_aggregator {
    LP_AGG_IDENTITY = 0,
    LP_AGG_SIGN = 1,
    LP_AGG_OPT = 2
} lp_aggregator;

typedef enum lp_ptr_space { LP_HOST = 0, LP_DEVICE = 1 } lp_ptr_space;

/* lp_solve flags */
#define LP_FLAG_RITZ   1u   /* finish with a Rayleigh-Ritz step: ordered basis + sigma */
#define LP_FLAG_TIMING 2u   /* record CUDA events around every fused power-step launch */
#define LP_FLAG_SIMT   4u   /* BF16 data: use the SIMT FP32 step kernel instead of the tensor-core one */
#define LP_FLAG_NO_GRAPH 16u     /* launch the solve's kernels one by one instead of replaying the
                                 * CUDA graph captured for this (k, schedule, aggregator, flags)  */
#define LP_FLAG_TRACE  32u   /* keep Z_t after every aggregation and the residual error rho_t
                             * (Def. 3) for lp_trace                                          */
#define LP_FLAG_TC_RESIDENT 8u  /* BF16 data: use the tensor-core step that keeps each tile in shared
                                 * memory for both contractions (cluster-split d) instead of the
                                 * streaming one; ignored for other dtypes */
#define LP_FLAG_KXK_FP64 64u /* the k x k work in FP64: the Gram matrix of CholQR2 (each FP32
                              * product summed in FP64) and its Cholesky factor, the k x k SVD
                              * of the Procrustes alignment (eq. (3)) and the eigen-solve of
                              * the final Rayleigh-Ritz step.  Without it these are FP32, with
                              * an FP64 Cholesky only where an FP32 pivot is too small; the
                              * d x k work (steps, triangular solves, averaging) is FP32
                              * either way.                                                   */

typedef struct lp_ctx lp_ctx;

typedef struct lp_stats {
    int32_t rounds;            /* aggregations performed = the paper's |I_T|          */
    int32_t local_steps;       /* sum of p_t (+1 for the Ritz pass)                   */
    int32_t step_launches;     /* launches of the fused power-step kernel             */
    int32_t k;
    int64_t n, d;
    int32_t m;
    int32_t path;              /* step kernel: 0 = SIMT FP32, 1 = tcgen05 with the tile resident in
                                * shared memory, 2 = tcgen05 streaming (second pass re-read from L2),
                                * 3 = tcgen05 pass-split pair (LP_KERNEL_PAIR)                        */
    double a_bytes;            /* algorithmic bytes of A read by the step kernels     */
    double ms_solve;           /* solve wall time on the stream (events)              */
    double ms_step_kernels;    /* summed step-kernel time (LP_FLAG_TIMING only)       */
    int32_t kernel_launches;   /* every kernel this solve launched                    */
    int32_t reserved;
} lp_stats;

/*
 * lp_create: open a context on `device`.
 *   hbm_budget_bytes: upper bound on device memory this context may allocate
 *                     (0 = no bound beyond what the device has).  Requests over
 *                     it fail with LP_ERR_OOM and allocate nothing.
 *   cuda_stream:      a cudaStream_t the context launches on (borrowed, must
 *                     outlive the context); NULL makes the context own a stream.
 * Ownership: *out belongs to the caller and is released with lp_destroy.
 */
lp_status lp_create(lp_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream);

/*
 * lp_load_partitions: copy the m row partitions A_i into library-owned device
 * memory (Sec. 2, DPI: A^T = [A_1^T, ..., A_m^T], A_i in R^{s_i x d}; the
 * weights are p_i = s_i / n with n = sum s_i).
 *   rows[m]        s_i >= 1.
 *   d              columns, d >= 1.
 *   parts[m]       pointer to partition i, s_i x d row-major, elements of `dtype`.
 *   row_scales[m]  LP_FP8_E4M3 only: s_i FP32 scales (value = code * scale); else NULL.
 *                  LP_F32_BF16X2 takes FP32 parts (like LP_F32) and splits them on the device.
 *   space          whether parts / row_scales are host or device pointers.
 * Replaces any previously loaded partitions.  The caller keeps its buffers.
 * New data of the same shapes (m, rows, d, dtype) are copied into the existing
 * device buffers: segment tables, kernel plans, tuning and captured solve graphs
 * stay valid, and only the copy costs time.  The previous solve's result is
 * invalidated either way (lp_result returns LP_ERR_STATE until the next solve).
 */
lp_status lp_load_partitions(lp_ctx* ctx, int m, const int64_t* rows, int64_t d, lp_dtype dtype,
                             const void* const* parts, const float* const* row_scales, lp_ptr_space space);

/*
 * lp_solve: run LocalPower (Alg. 1 with the aggregation of eqs. (3)-(4)) on the
 * loaded partitions.  Round t runs p_schedule[t] local power steps per
 * partition, Y_i <- (1/s_i) A_i^T (A_i Z_i) each followed (except the last) by
 * Z_i <- orth(Y_i), then one aggregation Y <- sum_i p_i Y_i D_i and Z <- orth(Y).
 * D_i = I whenever p_t = 1 (the remark after eq. (4)).  The base partition for
 * alignment is the one with the most rows (lowest index on ties).
 *   k              rank of the iterate (Alg. 1's iteration rank r >= the target
 *                  rank), 1 <= k <= min(LP_MAX_K, d, min_i s_i).  For a target
 *                  rank below k, use LP_FLAG_RITZ and take the leading columns.
 *   p_schedule[T]  p_t >= 1 (a decaying p is just a schedule, Sec. 3).
 *   y0             host pointer, d x k row-major FP64: the Gaussian start block
 *                  Y_0 (Alg. 1 initialisation); the library computes Z_0 = orth(Y_0).
 *   refine_rounds  extra p = 1 rounds appended after the schedule.
 *   flags          LP_FLAG_*.
 * Asynchronous on the context's stream; lp_result waits for it.
 */
lp_status lp_solve(lp_ctx* ctx, int k, const int* p_schedule, int T, lp_aggregator agg,
                   const double* y0, int refine_rounds, unsigned flags);

/*
 * lp_solve_seeded: lp_solve with the start block Y_0 drawn by the library from
 * `seed` instead of passed in (Alg. 1 starts from a random orthonormal basis;
 * Z_0 = orth(Y_0) as in lp_solve).  Y_0's d x k entries (row-major) are N(0,1)
 * draws from a counter-based generator: SplitMix64 (Steele, Lea & Flood, OOPSLA
 * 2014) evaluated at counters seed + (c + 1) * 0x9E3779B97F4A7C15, the top 53
 * bits as a uniform u in [0, 1), and Box-Muller on consecutive pairs: counters
 * 2q, 2q + 1 give r = sqrt(-2 ln(1 - u_2q)), theta = 2 pi u_2q+1, entry 2q =
 * r cos(theta) and entry 2q + 1 = r sin(theta).  The same seed gives the same
 * start on every machine up to the host's last-digit rounding of log, cos and
 * sin.  Same arguments, asynchrony and errors as lp_solve otherwise.
 */
lp_status lp_solve_seeded(lp_ctx* ctx, int k, const int* p_schedule, int T, lp_aggregator agg, uint64_t seed,
                          int refine_rounds, unsigned flags);

/*
 * lp_result: wait for the last solve and copy its output to host memory.
 *   z_out      d x k row-major FP64: Z_T = orth(Y_T) (Alg. 1 output), or with
 *              LP_FLAG_RITZ the Ritz vectors ordered by descending Ritz value.
 *              The basis is defined up to the sign of each column.  May be NULL.
 *   sigma_out  k values sqrt(n * lambda_j) (LP_FLAG_RITZ only; else zeros).  May be NULL.
 *   stats      may be NULL.
 * Returns LP_ERR_NUMERIC if a device-side check failed during the solve.
 */
lp_status lp_result(lp_ctx* ctx, double* z_out, double* sigma_out, lp_stats* stats);

/* Tuning of the streaming tensor-core step kernel (LP_BF16 and LP_F32_BF16X2
 * data).  Zero in a field keeps the library's default for it.  Ring depth, lag,
 * prefetch and cache hints change speed only: the same products are summed in
 * the same order.  slice_cols also changes how a tile's row products are
 * summed (over the CTAs of a cluster), so results can differ in the last bits. */
typedef struct lp_tuning {
    int32_t ring_units;      /* 32 KB shared-memory ring units (default: as many as fit, <= 8) */
    int32_t lag_units;       /* first-pass units of tile t+1 issued before the second pass of
                              * tile t starts (default 2 without a cluster, 4 with one)         */
    int32_t prefetch_units;  /* first-pass units brought into L2 ahead of their load (default 0) */
    int32_t cache_hints;     /* 1: first-pass loads mark lines evict_last, second-pass loads
                              * evict_first (default 0: no hint)                                  */
    int32_t slice_cols;      /* columns of A per CTA, a multiple of 128 (default: 1024 for one
                              * plane, 512 for two); smaller slices split d over a cluster and
                              * shorten the distance between a unit's HBM read and its L2 re-read */
    int32_t kernel;          /* LP_KERNEL_DEFAULT, LP_KERNEL_STREAM or LP_KERNEL_PAIR          */
    int32_t test_stall_cycles; /* test hook, 0 in normal use.  > 0: the pair kernel's HBM-pass
                              * producer, after its first ring fill, waits on a barrier that
                              * nothing completes, with this many SM clock cycles as the limit
                              * instead of the ~2 s of every other wait; the wait runs out, the
                              * kernel records the timeout, drains its copies and MMAs and
                              * returns, and the solve reports LP_ERR_TIMEOUT.  The context
                              * stays usable (reset the field and solve again).               */
} lp_tuning;

/* Tensor-core step kernels selectable through lp_tuning::kernel.
 * STREAM: one CTA per SM streams each 128-row tile through shared memory
 *         twice (the second time from L2) and forms both products.
 * PAIR:   the two passes run on the two CTAs of a cluster: rank 0 reads the
 *         tile from HBM and forms W = A_t Z, copies W into rank 1's shared
 *         memory, and rank 1 re-reads the tile from L2 and accumulates A_t^T W
 *         (d <= 1024 for k <= 16, d <= 512 for k > 16).  Same products, same
 *         summation order within a tile.
 * DEFAULT picks the pass-split pair kernel where it has a plan, else STREAM. */
enum { LP_KERNEL_DEFAULT = 0, LP_KERNEL_STREAM = 1, LP_KERNEL_PAIR = 2 };

/*
 * lp_set_tuning: set (tuning != NULL) or reset to defaults (NULL) the tuning
 * used by later lp_solve / lp_power_step calls on this context.  Negative
 * fields are LP_ERR_INVALID; a ring that does not fit shared memory is
 * clamped to what fits.
 */
lp_status lp_set_tuning(lp_ctx* ctx, const lp_tuning* tuning);

/*
 * lp_autotune: time the step-kernel candidates for rank k on the loaded
 * partitions and keep the fastest for later solves on this context (it sets
 * the context's tuning, and for LP_BF16 data whether the resident or the
 * streaming tensor-core kernel runs).  Candidates: the streaming kernel with
 * lag in {1, 2, 4}, cache hints off/on and the default or 512-column slices,
 * and the resident kernel where it has a plan.  Each is timed over 3 launches after a warm-up launch, on the
 * context's stream; the call synchronises.  Other dtypes have one candidate
 * (the SIMT kernel) and return at once.
 *   chosen      receives the winning tuning (may be NULL).
 *   path        receives the winning lp_stats::path code (may be NULL).
 *   best_ms     receives the winner's mean launch time in ms (may be NULL).
 */
lp_status lp_autotune(lp_ctx* ctx, int k, lp_tuning* chosen, int* path, double* best_ms);

/*
 * lp_trace: per-round records of the last solve run with LP_FLAG_TRACE
 * (synchronises the context's stream).
 *   z_trace  rounds x d x k FP64: Z_t = orth(Y_t) after round t's aggregation,
 *            row-major per round (may be NULL).
 *   rho      rounds values: rho_t = max_i ||Z_t^(i) G_i - Z_t^(b)||_2, the residual
 *            error of Def. 3 over the last local bases, G_i the solve's aligner
 *            (none for vanilla averaging); 0 in rounds with p_t = 1 (may be NULL).
 * rounds = T + refine_rounds of that solve.  LP_ERR_STATE without a traced solve.
 */
lp_status lp_trace(lp_ctx* ctx, double* z_trace, double* rho);

/*
 * lp_eta: the local-approximation measure of Def. 2 (Sec. 4) for the loaded
 * partitions, a property of the data that needs no solve:
 *   eta = max_i ||M_i - M||_2 / ||M||_2,  M_i = (1/s_i) A_i^T A_i,  M = sum_i p_i M_i.
 * Every M_i is formed on the device by ceil(d / 16) fused local power steps on
 * identity blocks of Z (the same step kernel and precision as a solve), M by a
 * p-weighted FP64 sum of the symmetrised M_i, and each spectral norm by a
 * Lanczos run of min(d, 256) steps with full reorthogonalisation (exact once
 * the run reaches d steps or an invariant subspace).
 *   eta    out: one double.
 *   norms  out, may be NULL: m + 1 doubles, ||M_i - M||_2 for i = 0 .. m-1, then ||M||_2.
 * Device memory: (m + 1) d^2 * 4 + (m + 1) * min(d, 256) * d * 4 bytes, within
 * the context's budget (LP_ERR_OOM otherwise), freed before the call returns.
 * Synchronous.  The last solve's result, statistics and status stay as they were.
 * Errors: LP_ERR_STATE (no partitions), LP_ERR_INVALID (eta NULL),
 * LP_ERR_UNSUPPORTED (no step kernel for d, or d > 16384), LP_ERR_NUMERIC
 * (M = 0 or a non-finite norm), LP_ERR_TIMEOUT (a bounded device wait gave up).
 */
lp_status lp_eta(lp_ctx* ctx, double* eta, double* norms);

/* lp_destroy: free everything the context owns; NULL is a no-op. */
void lp_destroy(lp_ctx* ctx);

/* lp_last_error: text of the last failure on this context ("" if none); valid
 * until the next call on the context.  With ctx == NULL: the last failure of a
 * call that has no context (lp_create, lp_power_step_static) on this thread. */
const char* lp_last_error(const lp_ctx* ctx);

/* ----------------------------------------------------------------------------
 * Request server: continuous batching of independent truncated-SVD solves on
 * one GPU.  The paper has no counterpart; it serves many LocalPower problems
 * at once.  Each admitted request gets its own context and stream, so its
 * partitions A_i and iterates Z_i stay on the device across its rounds while
 * the rounds of other requests run beside it; requests that arrive while
 * others run are admitted as soon as the HBM budget and the active-request
 * limit allow, in arrival order.  One thread drives a server at a time.
 * ------------------------------------------------------------------------- */
typedef struct lp_server lp_server;

typedef struct lp_request {
    /* the data, as for lp_load_partitions, plus a source row pitch */
    int m;
    const int64_t* rows;            /* m row counts s_i                                 */
    int64_t d;
    int64_t row_pitch;              /* elements between source rows (0 = d)            */
    lp_dtype dtype;
    const void* const* parts;       /* m pointers; must stay valid until completion    */
    const float* const* row_scales; /* LP_FP8_E4M3 only, else NULL                      */
    lp_ptr_space space;
    /* the solve, as for lp_solve */
    int k;
    const int* p_schedule;
    int T;
    lp_aggregator agg;
    const double* y0;               /* d x k row-major, host                           */
    int refine_rounds;
    unsigned flags;
} lp_request;

typedef struct lp_server_info {
    int64_t queued, active, completed;    /* requests by state (completed: not yet fetched) */
    uint64_t hbm_in_use, hbm_peak, hbm_budget;
} lp_server_info;

/*
 * lp_server_create: a server on `device` that admits requests while the sum of
 * their device-memory estimates stays within hbm_budget_bytes (0 = no bound)
 * and at most max_active (>= 1) are on the device.
 */
lp_status lp_server_create(lp_server** out, int device, size_t hbm_budget_bytes, int max_active);

/*
 * lp_server_submit: queue a request; *id receives its id (> 0).  The small
 * arrays (rows, p_schedule, y0, the pointer arrays) are copied; the partition
 * buffers are read when the request is admitted and must not change until it
 * completes.  LP_ERR_INVALID for malformed requests (the checks of
 * lp_load_partitions / lp_solve), LP_ERR_OOM when the request alone exceeds the
 * budget.
 */
lp_status lp_server_submit(lp_server* s, const lp_request* req, int64_t* id);

/*
 * lp_server_progress: retire requests whose solve finished (their device memory
 * is released), admit queued requests, and write up to `cap` ids of requests
 * that completed since the last call to done_ids (*n_done of them).  Admission
 * copies the partitions to the device and enqueues the whole solve on the
 * request's stream; nothing else waits for the GPU.
 */
lp_status lp_server_progress(lp_server* s, int64_t* done_ids, int cap, int* n_done);

/*
 * lp_server_result: results of a completed request (as lp_result), then the
 * request is forgotten.  Returns the request's own status (its load or solve
 * failure, if any); LP_ERR_STATE if the id is unknown or not complete.
 */
lp_status lp_server_result(lp_server* s, int64_t id, double* z_out, double* sigma_out, lp_stats* stats);

lp_status lp_server_query(lp_server* s, lp_server_info* info);

/* lp_server_error: text of the last failure on the server ("" if none). */
const char* lp_server_error(const lp_server* s);

/* lp_server_destroy: wait for active requests, free everything; NULL is a no-op. */
void lp_server_destroy(lp_server* s);

/* ----------------------------------------------------------------------------
 * Batch runner: many independent instances (the same lp_request description,
 * each its own shapes, schedule and dtype) loaded once and solved together by
 * one CUDA graph launch.  The paper has no counterpart.  Instances that share
 * the width d, the storage dtype, k, the schedule, the aggregator and the flags
 * form a group: their partitions are copied back to back into one group
 * context, and each step kind of the solve (the fused power step, the
 * reduction, the local and global CholQR2, the alignment, the aggregation, the
 * Rayleigh-Ritz pass) is one launch over all of the group's instances; the step kernel is persistent
 * (one CTA or CTA pair per SM walking the row pieces of every partition of
 * every instance).  The graph holds each group's whole solve as an independent
 * branch; it is captured on the first lp_batch_solve and replayed by later ones
 * until instances are added or re-tuned.  An instance's result depends on the
 * other instances of its group only through rounding (the row pieces follow the
 * group's rows), and replays reproduce it bit for bit.  A device error or a
 * numerical failure (LP_ERR_NUMERIC) in one instance is reported by every
 * instance of its group.  One thread drives a batch at a time.
 * ------------------------------------------------------------------------- */
typedef struct lp_batch lp_batch;

/* lp_batch_create: an empty batch on `device`; instances are admitted while
 * the sum of twice their device-memory estimates (each instance's data is held
 * as loaded and again in its group) stays within hbm_budget_bytes (0 = no
 * bound). */
lp_status lp_batch_create(lp_batch** out, int device, size_t hbm_budget_bytes);

/* lp_batch_add: load one instance (its partitions are copied to the device now;
 * the caller's buffers may be reused after the call); *index receives its
 * position.  LP_ERR_INVALID for malformed requests (LP_FLAG_TRACE included),
 * LP_ERR_OOM over budget. */
lp_status lp_batch_add(lp_batch* b, const lp_request* req, int* index);

/* lp_batch_autotune: form the groups now and lp_autotune each group's context
 * (the step kernel and its tuning chosen by timing on the group's own data);
 * groups formed later, after more instances are added, are tuned too. */
lp_status lp_batch_autotune(lp_batch* b);

/* lp_batch_solve: every instance's solve, asynchronously, as one graph launch. */
lp_status lp_batch_solve(lp_batch* b);

/* lp_batch_result: waits for the batch, then lp_result of instance `index`:
 * its basis and sigma; stats are its group's counters (rounds, launches, path,
 * timings) with this instance's n, m and A bytes. */
lp_status lp_batch_result(lp_batch* b, int index, double* z_out, double* sigma_out, lp_stats* stats);

/* lp_batch_size: number of instances (0 for NULL). */
int lp_batch_size(const lp_batch* b);

/* lp_batch_groups: number of groups the instances form (0 before the first
 * lp_batch_solve or lp_batch_autotune after an lp_batch_add, and for NULL). */
int lp_batch_groups(const lp_batch* b);

/* lp_batch_error: text of the last failure on the batch ("" if none). */
const char* lp_batch_error(const lp_batch* b);

/* lp_batch_destroy: wait for the batch and free everything; NULL is a no-op. */
void lp_batch_destroy(lp_batch* b);

/* ----------------------------------------------------------------------------
 * Single-kernel entry points, for checking one step of the method at a time.
 * They run on the context's stream and synchronise before returning.
 * ------------------------------------------------------------------------- */

/*
 * lp_power_step: one local power step for every loaded partition,
 * Y_i = (1/s_i) A_i^T (A_i Z_i) (eq. (2)).
 *   z      FP64 row-major; if z_shared, one d x k block used by every partition,
 *          else m consecutive d x k blocks (Z_1, ..., Z_m).
 *   y_out  m consecutive d x k FP64 blocks.
 *   space  where z and y_out live.
 * Synchronises the context's stream; LP_ERR_TIMEOUT if a bounded device wait
 * gave up (y_out is then not the product).
 */
lp_status lp_power_step(lp_ctx* ctx, int k, const double* z, int z_shared, double* y_out, lp_ptr_space space);

/*
 * lp_orth: Z_b = orth(Y_b) for a batch of `batch` d x k blocks (CholQR2: two
 * passes of Gram, Cholesky and triangular solve; eq. (1)'s orth, whose column
 * space is that of a Householder QR).  FP64 row-major in and out (`space`).
 * A block whose Gram matrix is not numerically positive definite yields
 * LP_ERR_NUMERIC.  flags: 0, or LP_FLAG_KXK_FP64 for the FP64 Gram and Cholesky.
 */
lp_status lp_orth(lp_ctx* ctx, int batch, int64_t d, int k, const double* y, double* z, lp_ptr_space space,
                  unsigned flags);

/*
 * lp_align_aggregate: Y = sum_i w_i Y_i D_i with D_b = I and D_i from `agg`
 * computed between Z_i and Z_b (eqs. (3)-(4); Alg. 1 aggregation).
 *   ys, zs   m consecutive d x k FP64 blocks each; w: m weights; base: b.
 *   y_out    d x k FP64; d_out (may be NULL) m consecutive k x k FP64 D_i.
 *   flags    0, or LP_FLAG_KXK_FP64 for the Procrustes SVD in FP64.
 */
lp_status lp_align_aggregate(lp_ctx* ctx, int m, int64_t d, int k, lp_aggregator agg, int base,
                             const double* w, const double* ys, const double* zs,
                             double* y_out, double* d_out, lp_ptr_space space, unsigned flags);

/* ----------------------------------------------------------------------------
 * Allocation-free entry point.  The paper has no counterpart: this call exists
 * for callers that cannot allocate device memory.
 * ------------------------------------------------------------------------- */

/*
 * lp_power_step_static: the local power step Y_i = (1/s_i) A_i^T (A_i Z) of
 * lp_power_step with one Z shared by every partition, run without any device
 * allocation and without a context.  It is meant for callers that must not
 * allocate: code running inside a memory pool or allocator it cannot re-enter,
 * a host that has reserved the device's memory up front, or a place where a
 * cudaMalloc would synchronise the device at the wrong moment.  Its scratch
 * (partial sums, row-segment table, padded Z and Y) lives in one 32 MiB array
 * inside the library, held on every GPU that loads the library until exit.
 *   A       device, FP32: the m partitions back to back, row-major, row pitch
 *           d; d a multiple of 4 and A 16-byte aligned.
 *   rows    host, m row counts s_i >= 1, with k <= min s_i.
 *   z       device, d x k FP64 row-major.
 *   y       device, m consecutive d x k FP64 blocks (output).
 *   stream  cudaStream_t to launch on (NULL: the legacy default stream).
 * Asynchronous: y holds the result once the stream passes this call's work.
 * A problem whose scratch would exceed the array fails with LP_ERR_INVALID
 * and launches nothing; lp_last_error(NULL) describes any failure.  The first
 * call on a device (made with that device current) looks up the array's
 * device address and keeps it for later calls.  Every call
 * shares the one array, which keeps the last call's contents: each call
 * writes everything it reads, but calls whose work overlaps on the GPU race.
 * A bounded wait that gives up inside the step kernel (a stall of seconds)
 * cannot be returned as a status by this asynchronous call; instead every
 * entry of y is set to NaN.
 */
lp_status lp_power_step_static(const float* A, int m, const int64_t* rows, int64_t d, int k, const double* z,
                               double* y, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LOCALPOWER_H */
