/*
 * pdot.h -- C ABI of the GB300 (sm_103a) PDOT library: restarted PDHG for
 * discrete optimal transport (arXiv 2407.19689).
 *
 * Problem (Eq. (1)):   min <C, X>   s.t.  X 1_n = f,  X^T 1_m = g,  X >= 0,
 * with C (m x n, non-negative), f (m) and g (n) probability vectors.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major: element (i, j) of C sits at C[i * ldc + j],
 *     0 <= i < m, 0 <= j < n, ldc >= n.  Plans passed in or out are dense
 *     row-major m x n (leading dimension n) in the handle's x_dtype.
 *   - Unless a name ends in _host, every pointer is a CUDA DEVICE pointer on
 *     the handle's device.  Inputs are borrowed for the duration of the call
 *     (for pdot_batch_submit: until pdot_poll reports the ticket).  The library
 *     owns its plan buffers, dual vectors and scratch memory, allocated with
 *     cudaMalloc and freed by pdot_destroy.
 *   - Work is issued on the handle's CUDA stream.  Every call returns only
 *     after its results are in place (it synchronises that stream), except
 *     pdot_batch_submit, which only queues.
 *   - Errors are reported only through return codes; nothing is thrown across
 *     the ABI.  A handle is used by one host thread at a time.
 *   - Calls that take a handle or a device index make that device the calling
 *     thread's current CUDA device (cudaSetDevice) and leave it so.
 *   - Argument errors (PDOT_ERR_ARG): m < 1, n < 1, ldc < n, tol <= 0 (solve),
 *     null required pointers, unknown dtypes, |sum f - sum g| > 1e-9 * max(sum f, 1)
 *     or a negative entry in f or g (checked on a host copy), x_dtype other
 *     than F32/F64, F64 plans with non-F64 costs or F32 plans with F64 costs.
 *     C is not scanned for negative entries.
 */
#ifndef PDOT_H
#define PDOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PDOT_OK = 0,
    PDOT_ERR_ARG = 1,
    PDOT_ERR_OOM = 2,
    PDOT_ERR_CUDA = 3,
    PDOT_ERR_NUMERIC = 4,    /* a KKT quantity became NaN or Inf */
    PDOT_MAX_ITER = 5,       /* pass budget spent; the last check's candidate is returned */
    PDOT_TIMEOUT = 6,        /* time_limit_s exceeded; the current iterate is returned */
    PDOT_BUSY = 7,           /* batch admission would exceed the HBM budget or slot count */
    PDOT_PENDING = 8,        /* ticket not finished yet */
    PDOT_CANCELLED = 9
} pdot_status;

typedef enum { PDOT_F32 = 0, PDOT_BF16 = 1, PDOT_F64 = 2, PDOT_POINTS = 3 } pdot_dtype;

/*
 * Cost generated on the fly (c_dtype = PDOT_POINTS).  Sec. 5.1 defines the
 * costs of its image workloads as distances between pixel coordinates; with
 * this form no m x n cost matrix exists: every pass computes
 *     C_ij = dist(xs_i, ys_j) / divisor
 * in FP32 from the coordinates (coordinate k = 0..d-1 accumulated in order,
 * then the quotient by the divisor's reciprocal with one FMA correction step,
 * the correctly rounded quotient on every value checked), which removes the
 * cost read from every plan pass (16 instead
 * of 20 bytes per plan entry) and the m x n cost buffer.  Any entry point that
 * takes (C, c_dtype, ldc) accepts it: C then points to a pdot_points_cost in
 * HOST memory (read during the call; pdot_batch_submit copies it), ldc is
 * ignored, and the plan must be FP32.  xs is m x d and ys is n x d, row-major
 * FP32, device memory (host memory for the _host entry points), borrowed like
 * C.  Errors (PDOT_ERR_ARG): d outside 1..8, an unknown dist, a null
 * coordinate pointer, divisor not finite and > 0, an FP64 plan.
 */
typedef enum { PDOT_DIST_SQEUCLID = 0, PDOT_DIST_L1 = 1, PDOT_DIST_L2 = 2, PDOT_DIST_LINF = 3 } pdot_dist;

typedef struct {
    int32_t d;              /* coordinates per point, 1..8 */
    pdot_dist dist;
    const float *xs;        /* m x d */
    const float *ys;        /* n x d */
    float divisor;          /* > 0 */
} pdot_points_cost;

/*
 * Solver options.  Defaults (pdot_default_options) follow Sec. 5 of the paper;
 * where the paper leaves a value open the default is a stated reading:
 *   tol 1e-4 (Sec. 5.1), restart check every 64 passes, adaptive step on
 *   (PDLP rule), adaptive restart on (beta_suff 0.1, beta_nec 0.9,
 *   beta_art 0.36), primal-weight update on (theta 0.5, omega0 1,
 *   eps_zero 1e-10), R = 1, scale-relative termination measures.
 * Theory mode (Algorithm 2 with the fixed-beta restart of Eq. (6) and the
 * constant step 1/(2 sqrt(m+n)) of Theorem 1): adaptive_step = 0,
 * adaptive_restart = 0, primal_weight_update = 0.
 */
typedef struct {
    double tol;                    /* relative KKT tolerance for termination */
    int64_t max_iter;              /* bound on PDHG passes (accepted + rejected) */
    double time_limit_s;           /* wall-clock limit of one solve, tested at chunk ends; <= 0: none.
                                      The solve then reports the current iterate with its own KKT
                                      measures (pdot_solve evaluates it after the chunk in flight; the
                                      batch engine stops the instance at its next restart check, where
                                      that iterate's measures are computed anyway) */
    int32_t restart_check_every;   /* K: restart/termination check after every K-th pass */
    int32_t adaptive_step;         /* 1: PDLP adaptive step size (Sec. 5); 0: constant eta */
    int32_t adaptive_restart;      /* 1: three restart conditions (Sec. 5); 0: Eq. (6) */
    int32_t primal_weight_update;  /* 1: PrimalWeightUpdate at restarts (Sec. 5) */
    double beta;                   /* decay of the fixed-beta restart, Eq. (6) */
    double beta_suff, beta_nec, beta_art;
    double theta;                  /* primal-weight smoothing */
    double eta0;                   /* initial/constant step; <= 0: 1/sqrt(m+n) adaptive, 1/(2 sqrt(m+n)) constant */
    double omega0;                 /* initial primal weight */
    double R;                      /* gap scaling in the KKT error (Sec. 3.1) */
    double eps_zero;               /* threshold of the primal-weight update */
    int32_t rel_mode;              /* 0: scale-relative termination measures; 1: cuPDLP "1 +" form */
    pdot_dtype x_dtype;            /* plan precision: PDOT_F32 (default) or PDOT_F64 */
    int32_t round_plan;            /* 1: return the Algorithm 3 rounding of the plan */
    int32_t use_graph;             /* 1: capture K-pass chunks as CUDA graphs (default) */
    int32_t tile_rows;             /* rows per plan tile (even, 2..4096); 0: pick by shape */
    uint64_t hbm_budget_bytes;     /* batch admission budget; 0: 90% of free memory at create */
    int32_t max_batch_slots;       /* most instances resident at once in the batch engine */
    int32_t chunk_checks;          /* check periods per batch chunk launch (serving granularity) */
    uint64_t batch_active_bytes;   /* 0: every resident batch instance advances in every chunk.  Otherwise
                                      a chunk advances the oldest resident instance, then younger ones in
                                      admission order whose per-pass plan bytes still fit this budget
                                      (large solves keep the bandwidth; small ones fill in beside them) */
    int32_t pass_kernel;           /* plan-pass kernel of single-instance calls with FP32 plans (pdot_solve,
                                      pdot_pdhg_steps, pdot_time_pass): 0 = the autotuner's choice (default),
                                      1 = register pipeline, 2 = bulk copies per row, 3 = bulk copies per
                                      4-row group (generated costs with d > 4 take 2 instead).  FP64 plans
                                      always take the register pipeline.  Other values: PDOT_ERR_ARG */
    int32_t compensated_cost;      /* FP32 plans (reading C9): 1 = the reduced cost C - p - q is formed
                                      from the FP64 duals split into FP32 hi/lo pairs, with the rounding
                                      error of C - p_hi recovered exactly (TwoSum), so its error is
                                      relative to itself rather than to p and q (far fewer passes where
                                      FP32 rounding would stall the solve; about 6 % more time per pass
                                      at 4096^2, 1 % at 16384^2, none where a pass is latency-bound);
                                      0 = (C - (float)p) - (float)q; 2 (default) = 1 for instances of
                                      fewer than 4M plan entries and in the batch engine, 0 above.
                                      No effect on FP64 plans.  Other values: PDOT_ERR_ARG */
    int32_t resident;              /* 1 = an instance with an FP32 plan and a stored FP32 / BF16 cost whose
                                      plan and average fit the shared memory of one thread-block cluster
                                      (8 CTAs; about 190k plan entries) runs in the resident kernel where
                                      pass_kernel and tile_rows are 0 (in the batch engine: where tile_rows
                                      is 0): the cluster keeps X and the average's deviation on chip and
                                      runs whole check periods of Algorithm 2 in one launch (pdot_solve,
                                      pdot_pdhg_steps and the batch engine); 0 (default) = the tile kernels
                                      for every instance (measured faster on one GB300 for single solves
                                      and for batches: the resident kernel computes an instance on 8 SMs
                                      and sweeps the plan twice per pass).  Other values: PDOT_ERR_ARG */
} pdot_options;

typedef struct {
    pdot_status status;
    double primal_obj;      /* <C, X> of the returned plan */
    double dual_obj;        /* f^T p + g^T q */
    double gap;             /* primal_obj - dual_obj */
    double kkt;             /* KKT error as printed in Sec. 3.1 (gap scaled by 1/R) */
    double rel_kkt;         /* max(rel_primal, rel_dual, rel_gap) */
    double rel_primal, rel_dual, rel_gap;
    int64_t iters;          /* accepted PDHG iterations */
    int64_t passes;         /* PDHG passes (accepted + rejected) */
    int64_t restarts;
    int64_t rejected_steps;
    double eta, omega;      /* final step size and primal weight */
    double seconds;         /* wall time of the call (batch: admission to completion) */
    double hbm_bytes;       /* algorithmic plan-pass bytes moved */
    double rounded_obj;     /* <C, X_feas> of Algorithm 3 when round_plan = 1, else NaN */
    int32_t returned_average; /* 1 if the returned iterate is the running average */
    int32_t tile_rows;      /* rows per plan tile the solve ran with (it fixes the FP32 summation
                               order: a solve with the same tile_rows option and pass kernel takes
                               the same passes and returns the same bits); 0 when it ran in the
                               resident kernel (whose order depends on the instance's shape only) */
} pdot_result;

typedef struct {
    double rp2;        /* ||X1 - f||^2 + ||X^T1 - g||^2 */
    double rd2;        /* ||[p 1^T + 1 q^T - C]^+||_F^2 */
    double cx;         /* <C, X> */
    double dual;       /* f^T p + g^T q */
    double gap;
    double kkt;
    double rel_p, rel_d, rel_gap, rel_kkt;
} pdot_kkt_parts;

typedef struct {
    int64_t m, n;
    const void *C;          /* device, m x ldc; or a host pdot_points_cost (c_dtype PDOT_POINTS) */
    pdot_dtype c_dtype;
    int64_t ldc;
    const double *f, *g;    /* device */
    double tol;             /* <= 0: the handle's tol */
    void *X_out;            /* nullable device, m x n in x_dtype */
    double *p_out, *q_out;  /* nullable device */
    uint64_t user_tag;
} pdot_request;

typedef struct pdot_handle pdot_handle;

/* Fill *opt with the defaults listed above. */
void pdot_default_options(pdot_options *opt);

/* Static string for a status code (never NULL). */
const char *pdot_status_str(pdot_status s);

/* Message of the last failed call on this handle ("" if none); valid until
 * the next call on the handle. */
const char *pdot_last_error(pdot_handle *h);

/* Create a solver handle on CUDA device `device`, issuing work on
 * `cuda_stream` (a cudaStream_t).  With NULL the handle creates its own
 * blocking stream, which the CUDA runtime orders with the legacy default
 * stream.  `opt` may be NULL (defaults).  *out receives the handle. */
pdot_status pdot_create(const pdot_options *opt, int device, void *cuda_stream, pdot_handle **out);

/* Free every buffer the handle owns.  Waits for its stream.  NULL is a no-op. */
pdot_status pdot_destroy(pdot_handle *h);

/*
 * Solve Eq. (1) with restarted PDHG (Algorithm 2 plus the Sec. 5 heuristics)
 * until the relative KKT error is <= tol (Sec. 5.1 termination).
 * C: device, dtype c_dtype (F32/BF16 with F32 plans, F64 with F64 plans), or
 * a host pdot_points_cost with c_dtype PDOT_POINTS (F32 plans).
 * f, g: device FP64.  X_out (m x n, x_dtype), p_out (m), q_out (n): nullable
 * device outputs of the returned iterate (or of its Algorithm 3 rounding for
 * X_out when round_plan = 1).  res: required.
 */
pdot_status pdot_solve(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                       const double *f, const double *g, double tol,
                       void *X_out, double *p_out, double *q_out, pdot_result *res);

/*
 * Starting point and solver state of pdot_solve_from.  Algorithm 2 takes an
 * initial point (X^{0,0}, p^{0,0}, q^{0,0}) as input; pdot_solve starts at the
 * origin (reading C1).  pdot_solve_from starts from a caller's point, or
 * resumes a solve from the state an earlier call exported (checkpoint /
 * resume: the paper has no counterpart).  All pointers are device memory.
 *   X0 (m x n, x_dtype), p0 (m), q0 (n): nullable initial point (a null part
 *       is 0).  The solve then runs exactly as pdot_solve does from there.
 *   state_in: nullable; pdot_state_bytes(m, n, x_dtype) bytes written as
 *       state_out by an earlier call on the same (m, n, x_dtype), the same C,
 *       f, g and the same options.  The solve continues from that state: the
 *       plans, duals, averages and restart anchor, the step size, primal
 *       weight and every counter.  A solve split at a stop by max_iter or
 *       time_limit_s and resumed this way takes the same passes and returns
 *       the same result, bit for bit, as the uninterrupted solve on a handle
 *       that picks the same pass kernel and tile height (the autotuner's
 *       choice is cached per handle; pass_kernel and tile_rows fix it).
 *       max_iter counts passes from the original start.  Overrides X0/p0/q0.
 *       A blob of another shape or type, or not written by this library:
 *       PDOT_ERR_ARG.
 *   state_out: nullable; receives the state when the solve stops (before the
 *       Algorithm 3 rounding of round_plan), whatever the status.
 */
typedef struct {
    const void *X0;
    const double *p0, *q0;
    const void *state_in;
    void *state_out;
} pdot_start;

/* Bytes of a solver-state blob for an m x n solve with plans in x_dtype
 * (F32 or F64); 0 for invalid arguments.  Needs no GPU. */
int64_t pdot_state_bytes(int64_t m, int64_t n, pdot_dtype x_dtype);

/* 1 if an m x n instance's FP32 plan and the average's deviation fit the
 * shared memory of one thread-block cluster of the resident kernel (8 CTAs,
 * rows split evenly; each CTA holds its rows of both at 4 B per entry plus
 * FP64 partial sums), else 0.  Whether such an instance runs resident also
 * depends on the options (pdot_options.resident) and its cost type.  Needs
 * no GPU. */
int32_t pdot_resident_fits(int64_t m, int64_t n);

/* pdot_solve from a starting point or a saved state (see pdot_start); start
 * may be NULL (then the same as pdot_solve). */
pdot_status pdot_solve_from(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                            const double *f, const double *g, double tol, const pdot_start *start,
                            void *X_out, double *p_out, double *q_out, pdot_result *res);

/* Same as pdot_solve with every pointer in HOST memory; the host <-> device
 * copies happen inside the call. */
pdot_status pdot_solve_host(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                            const double *f, const double *g, double tol,
                            void *X_out, double *p_out, double *q_out, pdot_result *res);

/*
 * k inner iterations of Algorithm 2 at constant step eta and primal weight
 * omega (tau = eta/omega, sigma = eta*omega), no restarts, starting from the
 * device state (X, p, q) and overwriting it with (X^k, p^k, q^k).  The uniform
 * running averages (Xbar, pbar, qbar) of Algorithm 2 are written when the
 * pointers are non-null.  k >= 0.  The plan pass is the kernel pdot_solve runs
 * for the same shape and cost type (the autotuner's choice, or the handle's
 * pass_kernel option), with the same tile height.
 */
pdot_status pdot_pdhg_steps(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                            const double *f, const double *g, int64_t k, double eta, double omega,
                            void *X, double *p, double *q, void *Xbar_out, double *pbar_out, double *qbar_out);

/* The KKT error of Sec. 3.1 at the device point (X, p, q), with the relative
 * measures of the handle's rel_mode and R; *out is host memory. */
pdot_status pdot_kkt(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                     const double *f, const double *g, const void *X, const double *p, const double *q,
                     pdot_kkt_parts *out);

/* Algorithm 3: write into X_out (device, m x n, x_dtype) the rounding of the
 * device plan X onto {X >= 0, X1 = f, X^T1 = g}.  X and X_out may alias.
 * A zero row/column sum keeps scale 1; a zero ||err_r||_1 skips the rank-one term. */
pdot_status pdot_round(pdot_handle *h, int64_t m, int64_t n, const void *X, const double *f, const double *g,
                       void *X_out);

/*
 * Certified lower bound on the optimum of Eq. (1) from a row dual p.  The
 * dual of Eq. (1) asks p_i + q_j <= C_ij (the constraint whose violation the
 * KKT error's dual term measures, Sec. 3.1); for a given p the largest such q
 * is q_j = min_i (C_ij - p_i), and weak duality gives
 *   lower = f^T p + g^T q <= OPT.
 * With the returned p of a solve (single or batched), `lower` and the
 * objective of the Algorithm 3 rounding of its plan (rounded_obj with
 * round_plan = 1, a feasible plan, so >= OPT) bracket the optimum: the
 * result's objective error is certified without an exact solver.  The paper
 * has no counterpart (it reports the duality gap of the rounded plan).
 *   C, c_dtype, ldc: as pdot_solve (a PDOT_POINTS descriptor included; the
 *   handle's x_dtype decides which cost types it accepts, as in pdot_solve);
 *   f (m), g (n), p (m): device FP64; q_out: nullable device output (n) of q;
 *   lower: HOST output.  The minimum is exact, so q is the same bits as the
 *   definition evaluated in FP64 on the same cost values; lower is an FP64
 *   sum in a fixed order.  Errors: PDOT_ERR_ARG for bad arguments (as
 *   pdot_solve, and a null p or lower), PDOT_ERR_OOM, PDOT_ERR_CUDA.
 */
pdot_status pdot_dual_bound(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                            const double *f, const double *g, const double *p, double *q_out, double *lower);

/*
 * Batch engine (continuous batching).  pdot_batch_submit queues `count`
 * requests and writes one ticket id per request; it never blocks on the GPU.
 * PDOT_BUSY: a request alone would exceed the HBM budget.  Requests wait in
 * the queue until memory and a slot are free.  pdot_poll advances the engine
 * (admits queued requests as memory frees up, launches the next chunk of
 * iterations for every resident instance, retires finished ones) and returns
 * up to `cap` finished tickets with their results; *n_done receives the
 * count.  pdot_poll never waits longer than one chunk.
 * pdot_cancel removes a queued or running ticket (reported by pdot_poll with
 * PDOT_CANCELLED).  Request pointers must stay valid until the ticket is
 * reported.
 */
pdot_status pdot_batch_submit(pdot_handle *h, const pdot_request *reqs, int count, uint64_t *ticket_ids);
pdot_status pdot_poll(pdot_handle *h, uint64_t *done_ids, pdot_result *done_results, int cap, int *n_done);
pdot_status pdot_cancel(pdot_handle *h, uint64_t ticket);
/* Counts of queued (not yet admitted) and resident instances. */
pdot_status pdot_batch_pending(pdot_handle *h, int *queued, int *running);

/*
 * Allocation-free Algorithm 3 rounding, for callers that cannot allocate
 * device memory when they need it (memory owned by another allocator, a
 * serving loop that forbids cudaMalloc/cudaFree after warm-up because they
 * synchronise the device, a plug-in inside an application that owns all
 * allocations).  Same result as pdot_round, but no handle and no allocation:
 * the scratch is a 3.7 MB array in the library's device image, held by every
 * GPU that loads the library until the process exits.  This entry point has
 * no counterpart in the paper.
 *   device: CUDA device to run on (made current); cuda_stream: stream to use
 *   (NULL = legacy default stream); X (m x n, x_dtype), f (m), g (n): device
 *   inputs; X_out: device output (may alias X).  Returns after the stream
 *   synchronises.
 *   Limits: 1 <= m, n <= 32768 and x_dtype F32 or F64, else PDOT_ERR_ARG.
 *   The first call on a device looks up the array's device address (once per
 *   device).  The address is kept for the life of the process, so calls on a
 *   device after a cudaDeviceReset of it are not supported.
 *   All calls share the one array: the library runs one call per device at
 *   a time (a lock held until the call's stream synchronises, on error paths
 *   too), so calls from several host threads or on several streams wait for
 *   each other instead of racing.  Each call writes every scratch word before
 *   reading it, so nothing carries over from the previous call.
 */
pdot_status pdot_round_noalloc(int device, void *cuda_stream, int64_t m, int64_t n, pdot_dtype x_dtype,
                               const void *X, const double *f, const double *g, void *X_out);

/* Kernel launches issued by this handle since creation (diagnostics). */
int64_t pdot_launch_count(pdot_handle *h);

/* Diagnostics for roofline measurement: set up the instance, take three
 * PDHG steps (so the running average is read), then launch the fused plan
 * pass `reps` times back to back on the handle's stream between two CUDA
 * events, each launch reading the plans the previous one wrote (as accepted
 * passes of a solve do; the dual update is left out, so every launch moves
 * the same bytes).  *ms_per_pass receives the mean device time of one pass;
 * *bytes_per_pass (nullable) the algorithmic bytes one pass moves:
 * m n (sizeof C + 4 sizeof X) (read C, X, Xbar; write X+, Xbar+; sizeof C
 * is 0 for a generated cost);
 * *kernel_variant (nullable) the pass kernel used for this shape: 0 register
 * pipeline, 1 bulk copies per row, 2 bulk copies per 4-row group (FP64 plans
 * always 0). */
pdot_status pdot_time_pass(pdot_handle *h, int64_t m, int64_t n, const void *C, pdot_dtype c_dtype, int64_t ldc,
                           const double *f, const double *g, int reps, double *ms_per_pass, double *bytes_per_pass,
                           int32_t *kernel_variant);

/*
 * Self-test of the failure path of the bulk-copy pass kernels: on `device`,
 * one warp waits, with their bounded wait, for a transfer that is announced on
 * a shared-memory barrier but never issued.  The wait gives up after `polls`
 * polls (1 .. 2^24) and *device_status (host memory) receives the status a
 * pass sets when a wait gives up: PDOT_ERR_CUDA (3).  Returns PDOT_OK when the
 * self-test ran, PDOT_ERR_ARG for a bad device, poll count or null pointer,
 * PDOT_ERR_CUDA on a CUDA error.  Nothing on the device traps or waits without
 * bound, and the CUDA context stays usable.
 */
pdot_status pdot_watchdog_selftest(int device, int64_t polls, int32_t *device_status);

#ifdef __cplusplus
}
#endif

#endif /* PDOT_H */
