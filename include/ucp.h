/*
 * ucp.h -- C ABI of libucp.so: the coordinate-descent sweep of the generic
 * UCP solver (Tseng, "A Generic Solver for Unconstrained Control Problems
 * with Integral Functional Objectives", ACC 2020) on Witsenhausen's
 * counterexample, computed by CUDA kernels for sm_103a (GB300).
 *
 * Problem (Section V-A): x1 = x0 + u0(x0), y1 = x1 + w, x2 = x1 - u1(y1),
 * J = E[k^2 u0^2 + x2^2], x0 ~ N(0, sigma^2), w ~ N(0, 1).  The library
 * carries the first controller as f(x0) = x1 = x0 + u0(x0) on the x0 grid and
 * u1 as a table U on the y grid, linearly interpolated and held constant
 * beyond its ends.  Controllers are step/linear tables on linearly spaced
 * samples as in Section III-D ("Initialization").
 *
 * One sweep (Algorithm 1's partial-exhaustion phase for m = 0, then the u1
 * update, then J):
 *   1. u0 step (Corollary 1, eq. (2), Section IV-A): for every x_i in
 *      parallel, f_i <- the first minimiser of
 *          g(u; x_i) = k^2 (u - x_i)^2 + sum_l phi_l (u - U^(u + w_l))^2
 *      over the candidate list [f_i; f_{i-r..i-1}, f_{i+1..i+r};
 *      n_coarse values symmetric about 0; n_levels levels of n_refine values
 *      around the best so far, each level n_refine/2 times finer].  Every
 *      x_i reads the pre-sweep f (Jacobi).
 *   2. u1 step: U_j <- E[x1 | y1 = y_j], the minimiser of the quadratic
 *      marginal cost C_1 (one Newton step of Section III-D; the closed form
 *      of Section IV-C).
 *   3. J <- sum_i p_i g(f_i; x_i) in FP64.
 * The same sweep solves zero-delay source-channel coding (Section V-B) when
 * ucp_params.problem = 1: f is u0 itself, g(u; x_i) = k^2 u^2 +
 * sum_l phi_l (U^(u + w_l) - x_i)^2 with equal weights phi_l, and the u1 step
 * is U_j <- E[x0 | x1 = y_j] under uniform noise (plain FP64 path).
 *
 * Conventions for every call:
 *   - Return value: a ucp_status.  No call aborts, traps or exits.  After
 *     UCP_E_CUDA or UCP_E_TIMEOUT the object is poisoned and later calls on
 *     it return UCP_E_STATE; ucp_last_error() gives a one-line reason.
 *   - Pointers named host_* or documented as host are host memory owned by
 *     the caller; the library copies from/to them before returning.  The
 *     library owns all device memory it allocates (through the context's
 *     allocator, or cudaMalloc if none was given) and frees it on destroy.
 *   - Objects are not thread-safe, except ucp_submit / ucp_poll, which may be
 *     called from any thread.
 *   - Device work is issued on the stream given at creation (cudaStream_t
 *     passed as void*; NULL is the CUDA default stream).
 */
#ifndef UCP_H
#define UCP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define UCP_API __attribute__((visibility("default")))
#else
#define UCP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    UCP_OK = 0,
    UCP_PENDING = 1,      /* ucp_poll: the request has not finished        */
    UCP_E_ARG = -1,       /* invalid argument; nothing was changed          */
    UCP_E_NOMEM = -2,     /* device allocation failed                       */
    UCP_E_BUDGET = -3,    /* one request alone exceeds the server budget    */
    UCP_E_CUDA = -4,      /* a CUDA call failed; the object is poisoned     */
    UCP_E_TIMEOUT = -5,   /* a bounded device wait gave up                  */
    UCP_E_STATE = -6,     /* object poisoned, destroyed or busy             */
    UCP_E_NOTFOUND = -7   /* unknown ticket                                 */
} ucp_status;

/* Problem and solver parameters (Section V-A problem; grids of Section
 * III-D).  All half widths must be multiples of delta (relative tolerance
 * 1e-9).  Grids: x_i = (i - X/delta) delta, i < 2X/delta + 1; likewise w and
 * y.  Prior weights p_i ~ exp(-x_i^2 / 2 sigma^2) and quadrature weights
 * phi_l ~ exp(-w_l^2 / 2) are normalised to sum 1 (rectangle rule). */
typedef struct {
    double k;           /* > 0                                              */
    double sigma;       /* > 0                                              */
    double delta;       /* > 0, common spacing of the x0, w and y grids     */
    double x_half;      /* x0 grid [-x_half, x_half]                        */
    double w_half;      /* w grid [-w_half, w_half]                         */
    double y_half;      /* u1 table grid [-y_half, y_half]                  */
    double cand_half;   /* coarse candidates cover [-cand_half, cand_half]  */
    int32_t n_coarse;   /* >= 2 (64)                                        */
    int32_t n_refine;   /* 2, 4, 8, 16 or 32 (16)                           */
    int32_t n_levels;   /* 0..8 (4)                                          */
    int32_t n_nbr;      /* neighbours per side, 0..8 (2: "2 points per
                           direction", Section III-D)                        */
    int32_t init_kind;  /* 0 identity f(x) = x (Section III-D);
                           1 odd staircase 3.5 sgn(x) (2 min(floor(|x|/7),2)+1);
                           2 table (init_table)                              */
    int32_t precision;  /* 0: plain FP64 path (every cost a sequential FP64
                           quadrature); 1: fast path (correlation tables
                           screen the candidates, near-ties re-decided by the
                           FP64 quadrature).  Both make the same decisions.  */
    const double* init_table; /* host, n_x values of f, init_kind 2 only     */
    uint64_t init_len;        /* must equal n_x for init_kind 2              */
    uint64_t flags;           /* reserved, must be 0                         */
    int32_t problem;    /* 0: Witsenhausen's counterexample (Section V-A):
                           x1 = x0 + u0(x0), y1 = x1 + w, w ~ N(0, 1),
                           J = E[k^2 u0^2 + (x1 - u1(y1))^2], f = x1.
                           1: zero-delay source-channel coding (Section V-B):
                           x1 = u0(x0) + w, w ~ U(-w_half, w_half),
                           J = E[k^2 u0^2 + (u1(x1) - x0)^2] (lambda = k^2),
                           f = u0; plain FP64 path only (precision 0).       */
    int32_t reserved;   /* must be 0                                         */
} ucp_params;

/* Device allocator hooks (e.g. a framework's caching allocator).  alloc
 * returns a device pointer aligned to 256 bytes or NULL. */
typedef void* (*ucp_alloc_fn)(size_t bytes, void* user);
typedef void (*ucp_free_fn)(void* ptr, void* user);

typedef struct ucp_ctx ucp_ctx;
typedef struct ucp_inst ucp_inst;
typedef struct ucp_batch ucp_batch;
typedef struct ucp_srv ucp_srv;

UCP_API const char* ucp_status_str(ucp_status s);
/* Reason for the last failing call on this thread (static storage). */
UCP_API const char* ucp_last_error(void);
/* Library version, build architecture string (e.g. "sm_103a"). */
UCP_API const char* ucp_version(void);

/* Validate params on the host without touching the GPU; returns the grid
 * sizes, the candidate-list length and the device bytes one instance will
 * hold (any output may be NULL).  UCP_E_ARG with ucp_last_error() naming
 * the offending field when invalid. */
UCP_API ucp_status ucp_plan(const ucp_params* params, uint64_t* n_x, uint64_t* n_w,
                            uint64_t* n_y, uint64_t* n_cand,
                            uint64_t* device_bytes);

/* Context: device ordinal, optional allocator (both NULL = cudaMalloc). */
UCP_API ucp_status ucp_ctx_create(int32_t device, ucp_alloc_fn alloc, ucp_free_fn free_fn,
                          void* user, ucp_ctx** out);
UCP_API ucp_status ucp_ctx_destroy(ucp_ctx* ctx);

/* ---- one instance ---------------------------------------------------- */

/* Validate params, build the grids and weights on the device, set f from
 * the init, then U <- E[x1 | y1] (problem 1: E[x0 | x1]) and J.  Work is
 * enqueued on `stream`. */
UCP_API ucp_status ucp_create(ucp_ctx* ctx, const ucp_params* params, void* stream,
                      ucp_inst** out);
/* Grid sizes, candidate-list length and device bytes held. */
UCP_API ucp_status ucp_sizes(const ucp_inst* inst, uint64_t* n_x, uint64_t* n_w,
                     uint64_t* n_y, uint64_t* n_cand, uint64_t* device_bytes);
/* Enqueue n_sweeps sweeps (asynchronous; J after each is recorded). */
UCP_API ucp_status ucp_sweep(ucp_inst* inst, int32_t n_sweeps);
/* Synchronise and return J of the current controllers. */
UCP_API ucp_status ucp_eval_J(ucp_inst* inst, double* J_out);
/* Synchronise and return J after each sweep: host out[0..n), out[0] is the
 * initial J; n is clamped to the sweeps done + 1, *n_written set. */
UCP_API ucp_status ucp_J_history(ucp_inst* inst, double* out, uint64_t n,
                         uint64_t* n_written);
/* Synchronise and copy the controllers to host buffers (any may be NULL):
 * f (n_x; u0 = f - x0 if as_paper_u0; problem 1 carries u0 itself, so f is
 * returned as is), U (n_y), idx = list position of the
 * winner of every x_i in the last sweep (n_x, -1 before the first sweep). */
UCP_API ucp_status ucp_get_controllers(ucp_inst* inst, double* f, uint64_t n_x,
                               double* u1, uint64_t n_y, int32_t as_paper_u0,
                               int32_t* idx);
/* Replace the state from host buffers: f (n_x values, rounded to the lattice
 * delta 2^-(n_levels log2(n_refine/2)) that all candidates lie on); U (n_y)
 * or NULL to recompute U (the u1 step of the instance's problem).  J is
 * recomputed.  Resume from a
 * checkpoint = ucp_get_controllers + ucp_set_controllers. */
UCP_API ucp_status ucp_set_controllers(ucp_inst* inst, const double* f, uint64_t n_x,
                               const double* u1, uint64_t n_y);
UCP_API ucp_status ucp_destroy(ucp_inst* inst);

/* ---- launch shapes (the autotuner's knobs) -------------------------------- */

/* How the same work is spread over threads; every valid choice gives the
 * same results, bit for bit (the arithmetic of every candidate cost, u1
 * target and reduction is fixed; only which thread runs it changes).  0 in
 * any field keeps the library's rule for it. */
typedef struct {
    int32_t search_lanes;   /* lanes per x0 point in the screened search:
                               4, 8 or 16 (rule: 8)                          */
    int32_t u1_threads[5];  /* threads sharing a u1 run of 1, 2, 4, 8, 16
                               targets: 1, 2 or 4, at most the run length
                               (rule: 4 for launches of at most 4 blocks per
                               SM and for runs of 16, else 1)                */
    int32_t defer_blocks;   /* blocks of the deferred near-tie search per
                               instance, 1..4096 (rule: one instance n_x/128
                               within [64, 4 per SM]; a batch of 16 or more
                               4 per instance, fewer 64 / n)                 */
} ucp_launch_config;

/* Set the launch shapes of later sweeps of an instance or a batch (captured
 * graphs are rebuilt; a batch synchronises its stream first), or, for a
 * context, the shapes that instances and batches created on it afterwards
 * start with.  UCP_E_ARG for a value outside its range. */
UCP_API ucp_status ucp_ctx_set_launch_config(ucp_ctx* ctx, const ucp_launch_config* cfg);
UCP_API ucp_status ucp_set_launch_config(ucp_inst* inst, const ucp_launch_config* cfg);
UCP_API ucp_status ucp_batch_set_launch_config(ucp_batch* b, const ucp_launch_config* cfg);

/* ---- one sweep split over processes (Section IV-A) ----------------------- */

/* For a fixed controller the u0 step of every x0 point is independent of
 * the others (Section IV-A), so one instance's sweep can be split over
 * processes (one per GPU): each holds the same instance, searches its range
 * of x0 points, the new values are exchanged, and every process finishes
 * the sweep (u1 step, tables, J) on the whole new controller.
 *   ucp_sweep_part: the search of x0 points i0 .. i1 - 1 (0 <= i0 <= i1 <=
 *     n_x) from the current state; f_part (host, i1 - i0 doubles) receives
 *     their new values.  Synchronises.  The winners' list positions
 *     (ucp_get_controllers idx) are valid for this range only.
 *   ucp_sweep_finish: f (host, n_x doubles) is the whole new controller
 *     (every range's part); it becomes the controller and the rest of the
 *     sweep runs, J recorded as after ucp_sweep.  Synchronises on the copy.
 * ucp_sweep_part over [0, n_x) followed by ucp_sweep_finish gives exactly
 * ucp_sweep(1).  UCP_E_ARG for ranges or buffers out of bounds. */
UCP_API ucp_status ucp_sweep_part(ucp_inst* inst, int64_t i0, int64_t i1, double* f_part);
UCP_API ucp_status ucp_sweep_finish(ucp_inst* inst, const double* f, uint64_t n_x);

/* ---- Algorithm 1's outer loop (Sections III-B to III-D) ----------------- */

/* Local update (Section III-D, "Local Update"): n iterations, each moving
 * every f_i (all x0 points in parallel, from the controller before the
 * iteration) by Newton's step on its marginal cost, u <- u - g'(u)/g''(u)
 * where g'' > 0, else by the gradient step u <- u - tau g'(u), the new value
 * rounded to the controller lattice (as ucp_set_controllers rounds a
 * table); then u1 <- its exact minimiser (the u1 step of ucp_sweep) and J,
 * recorded in the J history like a sweep.  g' and g'' are the derivatives of
 * the discretised cost, which is quadratic in u on each y-cell (from the
 * right at a cell boundary), formed by the w quadrature in FP64 in its fixed
 * order; g'' >= 2 k^2 > 0 on both problems, so the gradient branch is not
 * reached there.  The winners' list positions (ucp_get_controllers idx) keep
 * the last sweep's.  Asynchronous on the instance stream. */
UCP_API ucp_status ucp_local_update(ucp_inst* inst, int32_t n, double tau);

typedef struct {
    int32_t N;            /* iterations per round, >= 2 (20 in Section IV)    */
    int32_t max_rounds;   /* stop after this many rounds, >= 0               */
    double precision;     /* p >= 0: stop once I_L + I_P <= p (1e-10)        */
    double tau;           /* gradient step where g'' <= 0                    */
} ucp_solve_params;

typedef struct {
    int32_t rounds;            /* rounds run                                 */
    int32_t converged;         /* 1 if I_L + I_P <= p when the loop ended    */
    int32_t local_iters;       /* local-update iterations run                */
    int32_t exhaustion_iters;  /* partial-exhaustion iterations (sweeps) run */
    int32_t N_L, N_P;          /* the split the next round would take        */
    double J, I_L, I_P;        /* J at the end; the last round's changes     */
} ucp_solve_report;

/* Algorithm 1 ("Generic Solver") from the instance's current state: with
 * I_L = I_P = p and N_L = floor(N/2), N_P = N - N_L, while I_L + I_P > p:
 * N_L local-update iterations (ucp_local_update), I_L = |J before - J
 * after|; N_P partial-exhaustion iterations (ucp_sweep), I_P likewise; then
 * N_L = min(max(floor(I_L N / (I_L + I_P)), 1), N - 1), N_P = N - N_L
 * (the split kept when I_L + I_P = 0).  Synchronises after every phase to
 * read J.  J_phase (host, may be NULL, 1 + 2 max_rounds entries) receives
 * the starting J and J after every phase; NL_rounds (host, may be NULL,
 * max_rounds entries) N_L of every round run.  UCP_E_ARG for N < 2,
 * max_rounds < 0 or a negative or non-finite precision or tau. */
UCP_API ucp_status ucp_solve(ucp_inst* inst, const ucp_solve_params* params,
                             ucp_solve_report* report, double* J_phase,
                             int32_t* NL_rounds);

/* Fast path and problem 1's fast mode: number of candidate costs
 * re-computed by the fixed-order FP64 quadrature because screened table
 * costs left a near-tie open (since creation; 0 on the plain path).
 * Synchronises. */
UCP_API ucp_status ucp_tie_recosts(ucp_inst* inst, int64_t* out);

/* The fast path's correlation tables of the current u1 table, for tests and
 * diagnostics (Section V-A's w quadrature rewritten as three correlations of
 * E = U^(y) - y against the Gaussian weights: P_p = sum_l phi_l w_l E_{p+l},
 * Q_p = sum_l phi_l E_{p+l}^2, R_p = sum_l phi_l E_{p+l} E_{p+l+1}; E-index m
 * is y-index jlo + m, table position p covers candidate lattice cell
 * c_lo + p).  sizes (4 entries, required) receives n_pos, n_cols, c_lo and
 * jlo.  P, Q, R (host, n_pos entries each, may be NULL together) receive the
 * double-float table values as doubles; bound (host, n_cols entries, may be
 * NULL) the device's per-column bound on the error of S(u) = W2 +
 * 2[(1-t)P_p + t P_{p+1}] + (1-t)^2 Q_p + 2t(1-t) R_p + t^2 Q_{p+1} that the
 * tables cause at cells whose positions p, p + 1 lie in column p / 128.
 * UCP_E_ARG if a buffer is shorter than the instance's size, UCP_E_STATE on
 * the plain path.  Synchronises. */
UCP_API ucp_status ucp_get_tables(ucp_inst* inst, double* P, double* Q, double* R,
                                  int64_t n_pos, float* bound, int64_t n_cols,
                                  int64_t* sizes);

/* Work counters since creation (fast path; zeros on the plain path), the
 * first n of, in order:
 *   0 recosts     as ucp_tie_recosts;
 *   1 u1_pairs    (source, run of targets) pairs the u1 step summed directly;
 *   2 u1_boxes    (box of sources, run of targets) pairs it summed by the
 *                 boxes' Taylor expansions (pairs in neither were skipped as
 *                 negligible);
 *   3 u1_df_terms Taylor terms evaluated in double-float, over those box
 *                 pairs (per target of the run, each of two polynomials);
 *   4 u1_f32_terms Taylor terms evaluated in FP32, likewise;
 *   5 direct_costs candidate costs re-computed by the direct double-float
 *                 quadrature (the screening tier before ucp_tie_recosts).
 * out holds n >= 0 entries (n <= 6).  Synchronises. */
#define UCP_N_COUNTERS 6
UCP_API ucp_status ucp_work_counters(ucp_inst* inst, int64_t* out, int32_t n);

/* Per-kernel CUDA-event timing on the instance stream (off by default).
 * ucp_kernel_times fills up to cap entries: name (static), launches and
 * total milliseconds since the last reset; returns the entry count. */
UCP_API ucp_status ucp_profile(ucp_inst* inst, int32_t enable);
UCP_API int32_t ucp_kernel_times(ucp_inst* inst, const char** names,
                         int64_t* launches, double* total_ms, int32_t cap);

/* ---- batches ------------------------------------------------------------ */

/* Many instances swept together: params is a host array of n parameter sets
 * (different k, sigma, delta, grid widths and n_refine allowed; all
 * precision 1).  Each instance is set up as by ucp_create on `stream`;
 * a batched sweep then runs each kernel once for all instances (blocks mapped
 * to instances by a table) from a captured CUDA graph when `stream` is not
 * the default stream.  Every instance gets the same results as alone: the
 * kernels run the same per-instance arithmetic.  Section IV-A's independence
 * of the grid points within one controller update is what lets instances and
 * their grid points share one launch. */
UCP_API ucp_status ucp_batch_create(ucp_ctx* ctx, const ucp_params* params, int32_t n,
                                    void* stream, ucp_batch** out);
/* n_sweeps sweeps of every instance; returns when they are enqueued and the
 * host-side descriptors are consumed. */
UCP_API ucp_status ucp_batch_sweep(ucp_batch* b, int32_t n_sweeps);
/* Synchronise; J_out[k] = J of instance k (host array of n). */
UCP_API ucp_status ucp_batch_eval_J(ucp_batch* b, double* J_out);
/* Per-kernel CUDA-event timing of batched sweeps (off by default), as
 * ucp_profile / ucp_kernel_times for one instance: while on, batched sweeps
 * launch kernel by kernel (no graph replay) with events around each kernel
 * group (search, u1_boxes, u1_shift, mmse_main, mmse_combine, build_E,
 * tables, tab_combine, J); enabling resets the totals. */
UCP_API ucp_status ucp_batch_profile(ucp_batch* b, int32_t enable);
UCP_API int32_t ucp_batch_kernel_times(ucp_batch* b, const char** names,
                                       int64_t* launches, double* total_ms, int32_t cap);
/* Member k as an instance handle (for ucp_get_controllers, ucp_J_history,
 * ...); owned by the batch, valid until ucp_batch_destroy. */
UCP_API ucp_status ucp_batch_instance(ucp_batch* b, int32_t k, ucp_inst** out);
UCP_API ucp_status ucp_batch_destroy(ucp_batch* b);

/* ---- serving: continuous batching of solve requests ----------------------- */

/* Result of a served request (times in seconds since the server started). */
typedef struct {
    double J;            /* J after the last sweep                         */
    double t_submit;     /* ucp_submit returned                            */
    double t_admit;      /* admitted to a slot (set up on the GPU)         */
    double t_done;       /* results copied to host memory                  */
    int32_t sweeps;
    int32_t status;      /* ucp_status of the request                      */
} ucp_result;

typedef struct {
    int64_t queued;       /* submitted, waiting for a slot or for HBM      */
    int64_t in_flight;    /* admitted or done but not yet polled           */
    int64_t steps;        /* batched sweeps launched                       */
    int64_t completed;
    int32_t max_active;   /* most requests swept together so far           */
    uint64_t bytes_in_use;
    double now;           /* seconds since the server started              */
} ucp_srv_info;

/* Start a server on ctx's device: at most max_slots requests on the GPU at
 * once, and their device bytes (as ucp_plan reports, plus the J history)
 * within hbm_budget_bytes.  A server thread runs the steps on `stream`;
 * served instances take device memory from a pool owned by the server. */
UCP_API ucp_status ucp_srv_create(ucp_ctx* ctx, uint64_t hbm_budget_bytes,
                                  int32_t max_slots, void* stream, ucp_srv** out);
/* Queue one solve (params copied, including an init table) of n_sweeps
 * sweeps; never blocks.  UCP_E_BUDGET if the request alone exceeds the
 * budget; otherwise it waits for a slot and memory.  Thread-safe. */
UCP_API ucp_status ucp_submit(ucp_srv* s, const ucp_params* params, int32_t n_sweeps,
                              uint64_t* ticket);
/* UCP_PENDING until the request is done; then fills res (may be NULL) and
 * the host buffers f (n_x) and u1 (n_y) (either may be NULL), forgets the
 * ticket and returns the request's status.  UCP_E_NOTFOUND for an unknown
 * or already collected ticket.  Thread-safe. */
UCP_API ucp_status ucp_poll(ucp_srv* s, uint64_t ticket, ucp_result* res, double* f,
                            uint64_t n_x, double* u1, uint64_t n_y);
UCP_API ucp_status ucp_srv_stats(ucp_srv* s, ucp_srv_info* info);
/* Failure drill on the host: the next step fails as a launch would (every
 * request in flight and queued ends with UCP_E_CUDA, later submissions get
 * UCP_E_STATE).  No device fault is involved. */
UCP_API ucp_status ucp_srv_fail_next_step(ucp_srv* s);
/* Stop the server thread and free everything; UCP_E_STATE if requests were
 * still pending (they are discarded), else UCP_OK. */
UCP_API ucp_status ucp_srv_destroy(ucp_srv* s);

/* Test hook of the bounded waits (no paper counterpart): with on = 1 the
 * tensor-core table kernel of this fast-path instance no longer issues its
 * filter-slice copy, so the one wait that copy would complete runs out (after
 * a short bound; nothing is in flight behind it).  With on = 2 its builder
 * warps stop after the first filter tile, so the MMA thread's wait for the
 * second runs out (short bound) while the first slice group's MMAs are in
 * flight; it waits for them to complete.  Either way the kernel then waits
 * for its copies, writes zero partials, frees its tensor memory and sets the
 * error flag; the next synchronising call returns UCP_E_TIMEOUT and the
 * instance is poisoned.  on = 0 restores normal operation; other values get
 * UCP_E_ARG.  UCP_E_STATE on the plain path. */
UCP_API ucp_status ucp_test_tc_skip_copy(ucp_inst* inst, int32_t on);

/* Measured ALU throughput of the current device (no paper counterpart: the
 * denominators of the roofline fractions of the ALU-bound kernels): FP64
 * FMA and FP32 FMA in TFLOP/s (2 flops per FMA) and FP32 ex2 (SFU) in
 * Gop/s, from dependent-chain kernels that fill every SM.  Allocates and
 * frees a small device buffer; synchronises. */
UCP_API ucp_status ucp_probe_alu(double* fp64_tflops, double* fp32_tflops,
                                 double* ex2_gops, void* stream);

/* ---- allocation-free u1 step ------------------------------------------- */

/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory (a process whose device memory is owned by
 * another framework, a real-time control loop that must not enter the
 * allocator, a plug-in handed only its input and output buffers).
 *
 * Computes the u1 table U_j = E[x1 | y1 = y_j] (the same u1 step as
 * ucp_sweep / ucp_set_controllers on the fast path) for the controller f:
 *   params  host; validated as by ucp_plan (precision is ignored).
 *   f_dev   device, n_x doubles: f(x_i) on the x0 grid, rounded to the
 *           candidate lattice as ucp_set_controllers does.
 *   u1_dev  device, n_y doubles, written.
 *   stream  cudaStream_t as void* (NULL: default stream); the call is
 *           asynchronous on it.
 * It allocates nothing: its intermediate buffers live in one fixed device
 * array of 5.9 MiB that every GPU loading the library holds until exit.
 * Limits: n_x <= 32768 and n_y <= 32768, else UCP_E_ARG.  Each call outside
 * stream capture looks up that array's address with the device current (so
 * the call stays valid after cudaDeviceReset); a call while `stream` is
 * capturing uses the address of the last uncaptured call on the device, and
 * UCP_E_STATE if there was none -- make one call before capturing.  All
 * calls share the array: calls that overlap on the GPU race, so serialise
 * them.  UCP_E_CUDA on a launch failure. */
UCP_API ucp_status ucp_u1_update_noalloc(const ucp_params* params,
                                         const double* f_dev, double* u1_dev,
                                         void* stream);

/* ---- the 2-dimensional Witsenhausen counterexample (Section V-D) -------- */

/* The state, both controllers and the observation are vectors in R^2:
 *   x1 = x0 + u0(x0),  y1 = x1 + w,  x2 = x1 - u1(y1),
 *   J = (1/2) E[k^2 |u0|^2 + |x2|^2],  x0 ~ N(0, sigma^2 I),  w ~ N(0, I)
 * (the factor 1/2 makes J per dimension, so that it compares with the
 * scalar problem's).  The sweep is the scalar one in two dimensions, in FP64
 * with every sum in a fixed order:
 *   - u0 step, for every x0 point the first minimiser of
 *     g(u; x) = k^2 |u - x|^2 + sum_cd phi_c phi_d |u - U^(u + w_cd)|^2
 *     (U^ the bilinear interpolant of the u1 tables, held constant beyond
 *     them) over the candidate list: the incumbent; f at the other points of
 *     the (2 n_nbr + 1)^2 window around the point (the incumbent where the
 *     window leaves the grid); the n_coarse x n_coarse coarse grid
 *     c_j = (2j - (n_coarse - 1)) (q/2) delta per axis, q = 2 ceil(cand_half /
 *     ((n_coarse - 1) delta)); then n_levels levels of the 8 neighbours
 *     best + (s, t) q delta 2^-level, (s, t) in {-1, 0, 1}^2 \ (0, 0) in
 *     row-major order, around the best so far;
 *   - u1 step, U(y) = E[x1 | y1 = y] per component (Section IV-C);
 *   - J in index order.
 * Grids: one spacing delta for x0 (n_x x n_x points over [-x_half,
 * x_half]^2), w (n_w x n_w over [-w_half, w_half]^2) and y (n_y x n_y);
 * point (a, b) is ((a - h) delta, (b - h) delta) with flat index a n + b.
 * Controller values lie on the lattice delta 2^-n_levels Z per component. */
typedef struct {
    double k, sigma, delta;
    double x_half, w_half, y_half, cand_half;   /* multiples of delta          */
    int32_t n_coarse;   /* coarse values per axis, 2..64                       */
    int32_t n_levels;   /* refinement levels, 0..40                            */
    int32_t n_nbr;      /* window radius, 0..8                                 */
    int32_t direct;     /* bit 0 clear: screened search (correlation tables of
                           u1 with a certified error bound, the exact quadrature
                           only for candidates the bound cannot separate) and J
                           from the same tables (within half the prior-weighted
                           bound, ~1e-10, of the exact J); set: the exact
                           quadrature for every candidate (same decisions) and
                           for J.  Bit 1 clear: the u1 weights factorised
                           per axis (GEMM-shaped sums); set: each weight's
                           exponential formed directly (u1 equal to rounding). */
} ucp2_params;

typedef struct ucp_inst2 ucp_inst2;

/* Sizes per axis and the candidate-list length (outputs may be NULL).
 * UCP_E_ARG when params are invalid or the grids exceed n_x <= 441,
 * n_y <= 2049, n_w <= 1025. */
UCP_API ucp_status ucp2_plan(const ucp2_params* params, uint64_t* n_x, uint64_t* n_w,
                             uint64_t* n_y, uint64_t* n_cand);
/* New instance on `stream` (cudaStream_t as void*): the weights, the start
 * (init_f NULL: the identity f(x) = x of Section III-D; else host, n_x^2
 * pairs f[2 i + k], rounded to the lattice), its u1 step and J as entry 0
 * of the J history.  Device memory comes from the context's allocator. */
UCP_API ucp_status ucp2_create(ucp_ctx* ctx, const ucp2_params* params,
                               const double* init_f, void* stream, ucp_inst2** out);
/* n sweeps (u0 step, u1 step, J), asynchronous on the instance's stream. */
UCP_API ucp_status ucp2_sweep(ucp_inst2* inst, int32_t n);
/* J after 0, 1, ... sweeps into host `out` (at most n entries). */
UCP_API ucp_status ucp2_J_history(ucp_inst2* inst, double* out, uint64_t n,
                                  uint64_t* n_written);
/* Host copies (each may be NULL; lengths in elements): f (2 n_x^2,
 * f[2 i + k]), the u1 tables (2 n_y^2, U[2 t + k]) and the winners' list
 * positions of the last sweep (n_x^2; -1 before the first sweep).  UCP_E_ARG
 * if a buffer is shorter than that. */
UCP_API ucp_status ucp2_get_controllers(ucp_inst2* inst, double* f, uint64_t f_len,
                                        double* u1, uint64_t u1_len, int32_t* idx,
                                        uint64_t idx_len);
/* Replace f (host, 2 n_x^2 values, rounded to the lattice) and, when u1 is
 * not NULL, the u1 tables (2 n_y^2); with u1 NULL the u1 step runs.  J is
 * recomputed into the history's current entry.  UCP_E_ARG for other lengths
 * or values beyond the lattice's range. */
UCP_API ucp_status ucp2_set_controllers(ucp_inst2* inst, const double* f, uint64_t f_len,
                                        const double* u1, uint64_t u1_len);
/* Per-kernel-group CUDA-event timing of later sweeps (enable 1; 0 stops
 * and clears), read by ucp2_kernel_times as for ucp_kernel_times: up to cap
 * entries of a static group name, its launches and total milliseconds;
 * returns the number of groups, -1 on error.  Synchronises. */
UCP_API ucp_status ucp2_profile(ucp_inst2* inst, int32_t enable);
UCP_API int32_t ucp2_kernel_times(ucp_inst2* inst, const char** names, int64_t* launches,
                                  double* total_ms, int32_t cap);
/* Work counter since creation: (target, source) pair slots the factorised
 * u1 sums evaluated -- 32 sources x 32 x 32 targets per stage not skipped as
 * negligible, padding at the grid's edges included.  Synchronises. */
UCP_API ucp_status ucp2_work_counters(ucp_inst2* inst, int64_t* live_pairs);
UCP_API ucp_status ucp2_destroy(ucp_inst2* inst);

#ifdef __cplusplus
}
#endif
#endif
