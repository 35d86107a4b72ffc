/* hprqp.h — C ABI of the GB300 (sm_103a) HPR-QP library.
 *
 * HPR-QP (arXiv 2507.02470) solves the convex composite quadratic program of Sec. 1,
 * eq. (1.1):
 *
 *     min_x  1/2 <x, Q x> + <c, x> + phi(x)      s.t.   l <= A x <= u,
 *
 * where Q is symmetric positive semidefinite and may be given only as an operator, A is a
 * sparse m x n matrix, and phi is the indicator of the box C = [L, U] (the CQP of eq. (1.2)),
 * lambda * ||x||_1, or both.  The method is the dual Halpern Peaceman–Rachford iteration of
 * Algorithm 4 with the restart rules (3.6)–(3.8) and the sigma update of Algorithm 5, run
 * entirely in FP64 on the GPU.
 *
 * Conventions for every entry point:
 *   - Pointers to problem data may point to host memory or to device memory of the current
 *     CUDA device; the library detects which (cudaPointerGetAttributes) and copies.
 *   - Infinite bounds are IEEE +-INFINITY: l, L may be -INFINITY and u, U +INFINITY
 *     (Sec. 1); l = +INFINITY or u = -INFINITY (an empty row set), L = +INFINITY or
 *     U = -INFINITY are errors.  NaN anywhere in the data is an error.
 *   - Index arrays are int32, CSR row pointers start at 0 and are non-decreasing, column
 *     indices lie in [0, ncols).  Row entries need not be sorted.
 *   - Functions never abort or exit; they return a status and, on failure, record a message
 *     readable with hprqp_last_error().  A failed call leaves the handle usable.
 *   - A handle is not thread-safe: calls on one handle must be serialised by the caller.
 */
#ifndef HPRQP_H
#define HPRQP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hprqp_status {
  HPRQP_OK = 0,              /* converged: max(eta_p, eta_d, eta_gap) <= tol (Sec. 4.1) */
  HPRQP_MAX_ITER = 1,        /* iteration limit reached; the last bar iterate is kept */
  HPRQP_TIME_LIMIT = 2,      /* wall-clock limit reached */
  HPRQP_NUMERICAL_ERROR = 3, /* NaN/Inf appeared in the iteration or its residuals */
  HPRQP_INVALID_ARG = 4,     /* bad sizes, bounds with l > u, L > U or an infinite bound on
                                the wrong side, NaN, bad CSR */
  HPRQP_CUDA_ERROR = 5,      /* a CUDA runtime call failed (message in last_error) */
  HPRQP_TIMEOUT = 6,         /* a bounded device wait gave up (batched queue) */
  HPRQP_OOM = 7              /* device allocation failed */
} hprqp_status;

/* Kinds of additive Q terms (Sec. 1: Q need not be an explicit matrix). */
typedef enum hprqp_qkind {
  HPRQP_Q_DIAG = 1,          /* Q += diag(dense[0..n))                                   */
  HPRQP_Q_CSR = 2,           /* Q += n x n CSR matrix (rowptr, colidx, vals), symmetric   */
  HPRQP_Q_DIA = 3,           /* Q += symmetric band: offsets[k] >= 0, diags is ndiag x n,
                                diags[k*n + i] = Q[i][i + offsets[k]] (entries with
                                i + offsets[k] >= n are ignored)                          */
  HPRQP_Q_FACTOR = 4,        /* Q += B^T B, B a p x n CSR matrix (matrix-free)            */
  HPRQP_Q_DENSE_FACTOR = 5,  /* Q += F^T F, F a dense row-major p x n matrix              */
  HPRQP_Q_QAP = 6            /* Q vec(X) += vec(Ahat X Bhat - S X - X T) for d x d X with
                                n = d^2, vec(X)[i + j d] = X[i][j] (the QAP relaxation of
                                Sec. 4.5): p = d, dense = Ahat, Bhat, S, T (symmetric d x d,
                                4 d^2 values one after another); applied as two FP64
                                contractions, Ahat X then [Ahat X | S | X][Bhat; -X; -T];
                                at most one such term; not with launch_mode 3 */
} hprqp_qkind;

typedef enum hprqp_phi {
  HPRQP_PHI_BOX = 0,         /* phi = indicator of C = [L, U] (eq. (1.2))                */
  HPRQP_PHI_L1 = 1,          /* phi = lambda ||x||_1 (Lasso, Sec. 4.4); L, U ignored     */
  HPRQP_PHI_L1_BOX = 2       /* phi = lambda ||x||_1 + indicator of [L, U]               */
} hprqp_phi;

typedef struct hprqp_qterm {
  int32_t kind;              /* hprqp_qkind */
  int64_t p;                 /* FACTOR / DENSE_FACTOR: number of rows of B or F */
  int64_t nnz;               /* CSR / FACTOR: number of stored entries */
  const int32_t* rowptr;     /* CSR: n+1; FACTOR: p+1 */
  const int32_t* colidx;     /* CSR / FACTOR: nnz */
  const double* vals;        /* CSR / FACTOR: nnz */
  int32_t ndiag;             /* DIA: number of stored diagonals (<= 8) */
  const int32_t* offsets;    /* DIA: ndiag offsets, distinct, >= 0 */
  const double* diags;       /* DIA: ndiag x n */
  const double* dense;       /* DIAG: n values; DENSE_FACTOR: p x n row-major */
} hprqp_qterm;

/* Q as a sum of terms; nterms == 0 means Q = 0 (the LP case of the Sec. 2.2 remark). */
typedef struct hprqp_qop {
  int32_t nterms;
  const hprqp_qterm* terms;
} hprqp_qop;

/* Allocator hooks (optional): if alloc is non-NULL all device memory of the handle is
 * obtained from alloc(bytes, ctx, stream) and returned with free(ptr, bytes, ctx, stream). */
typedef void* (*hprqp_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*hprqp_free_fn)(void* ptr, size_t bytes, void* ctx, void* stream);

typedef struct hprqp_params {
  void* stream;              /* cudaStream_t for all work (the power method on A A^* runs on
                                an internal stream forked from and joined back to it); NULL:
                                the handle creates one */
  int64_t check_every;       /* termination test period, default 100 (Table 1 counts) */
  int64_t restart_every;     /* restart test period (R~ evaluation), default 10 */
  double alpha1, alpha2, alpha3;   /* restart parameters, defaults 0.2, 0.8, 0.5 (Sec. 4.1) */
  double alpha3_tight;       /* alpha3 after the residual ratio drops to ratio_tight: 0.2 */
  double ratio_tight;        /* 0.1 (Sec. 4.1) */
  double lambda_A;           /* > 0: use as lambda_A >= lambda_1(AA^*); else power method */
  double lambda_Q;           /* > 0: use as lambda_Q >= lambda_1(Q);    else power method */
  double sigma0;             /* > 0: initial sigma; else ||b||/||c|| rule of Sec. 4.1 */
  int64_t power_max_iter;    /* power method cap, default 5000 */
  double power_tol;          /* relative change of the Rayleigh quotient, default 1e-6 */
  double power_safety;       /* lambda = safety * estimate, default 1.01 */
  int32_t halpern_total;     /* 1: Halpern weight 1/(k+2) from the total counter (Alg. 4
                                as printed); 0 (default): inner counter t */
  int32_t sigma_golden;      /* 1: golden-section search for eq. (3.12); 0: exact argmin */
  int32_t restart_off;       /* 1: no restarts (Algorithm 3 with fixed sigma) */
  int32_t sigma_fixed;       /* 1: keep sigma0 at restarts */
  double time_limit;         /* seconds, <= 0: none (Sec. 4.1 uses 3600) */
  int32_t iters_per_launch;  /* iterations captured per CUDA-graph launch, default 64 */
  int32_t autotune;          /* 1 (default): time the SpMV schedules (lanes per row 1-32,
                                the staged form that streams a chunk's entries as one range,
                                or for A and A^T a SELL-32 copy) at create and pick the
                                fastest for each operator;
                                0: lanes per row from the mean row length; 2: the staged
                                form for every CSR pass; 3: the SELL-32 copy for the A and
                                A^T passes (rows sorted by length inside each 256-row chunk,
                                one row per lane), one lane per row elsewhere */
  int32_t verbose;           /* 0: silent; 2: wall time of each phase of hprqp_create, and the
                                batched autotuner's timings, on stderr */
  hprqp_alloc_fn alloc;      /* optional allocator hooks (see above) */
  hprqp_free_fn free;
  void* alloc_ctx;
  int32_t launch_mode;       /* 0 (default): CUDA graphs with conditional nodes: whole check
                                periods through a graph whose step variants are fixed by
                                position (see fixed_schedule), the rest through a graph whose
                                conditional nodes pick each step's variant on the device;
                                1: graph without conditional nodes (variants read at run time
                                inside the kernels);
                                2: plain stream launches of the same step variants, chosen on
                                the host after each step (for profilers that cannot follow
                                conditional graph nodes; one host synchronisation per step);
                                3: persistent solver, all passes of up to 4096 inner steps in
                                one cooperative launch with grid barriers between passes (one
                                launch per solve segment; slower than mode 0 on every
                                configuration measured) */
  int32_t scaling;           /* 1 (default): the Sec. 4.1 preconditioning (10 Ruiz passes, then
                                Pock-Chambolle with alpha = 1, on K = [Q A^T; A 0]) when Q is
                                explicit (DIAG, CSR and DIA terms only) and phi is the box
                                indicator; the iteration runs on the scaled problem while the
                                stopping test, hprqp_get, hprqp_apply and warm starts stay in
                                the original variables.  0: never scale. */
  int32_t method;            /* 0 (default): HPR-QP, Algorithm 4.  1, 2: the primal HPR methods of
                                Appendix A (Algorithm 6 on reformulation (1.3), Algorithm 7 on
                                (1.4)), for ablations: fixed sigma (sigma0 or the Sec. 4.1 rule),
                                no restarts, stopping rule of Sec. 4.1 every check_every steps;
                                they need scaling = 0 and run as stream launches */
  int32_t pdl;               /* 1 (default): consecutive kernels of a step are programmatic
                                dependent launches (a kernel's launch overlaps the end of the
                                one before it; results unchanged); 0: ordinary launches */
  int32_t fixed_schedule;    /* 1 (default, launch_mode 0): while a whole period remains, run
                                graphs whose step variants are fixed by position (R~ test every
                                restart_every, stopping test every check_every steps) with one
                                conditional node per R~ test instead of two per step; results
                                unchanged.  0: every step through the dynamic graph */
  int32_t tiled_factor;      /* factor terms B_f^T B_f: 1 (default) a large factor (>= 2e6
                                entries, >= 8 per row and column) also gets a copy stored tile
                                by tile, and the one-vector products B_f x, B_f^T t gather from
                                shared-memory tiles; 2: every factor that fits (n up to 64
                                tiles of 25,600 columns, p up to 8 tiles); 0: never.  Not with
                                launch_mode 3.  Sums in another order (rounding only) */
  int32_t fused_steps;       /* 1 (default; fixed-schedule graph, Q and A present): a plain step
                                followed by a Halpern step ends with two fused passes, A^T ybar
                                with the Halpern update of (w_Q, A^* y), then Q w of the new
                                iterate with the next step's elementwise pass of eqs. (3.1)-(3.3),
                                so that step runs no separate elementwise kernel; Q w is then
                                formed directly instead of by the Halpern recurrence of its
                                image (rounding only).  0: every step runs all five passes */
  int32_t factor_inline;     /* factor terms B_f^T B_f without a tiled copy: 1 (default) a thin
                                factor (sum over B's rows of their squared lengths <= n / 2)
                                has the inner step's products t = B x formed inside the Q row
                                pass from B's rows, with no separate pre-pass launch; 2: every
                                such factor; 0: never.  Sums in another order (rounding only) */
  int32_t wait_polls;        /* launch_mode 3: polls of one grid-barrier wait before the solve
                                gives up with HPRQP_TIMEOUT; 0 (default): about a second */
  int32_t batch_team;        /* batched solver: 0 (default) threads per instance chosen per bucket
                                of n (autotune 1: timed on the batch; 0: 512/256/128/64 from the
                                largest n down); 64, 128, 256 or 512: that block size for all */
} hprqp_params;

/* Residuals at the returned bar iterate (Sec. 4.1) and solve statistics. */
typedef struct hprqp_kkt {
  double eta_p, eta_d, eta_gap, rel_kkt; /* rel_kkt = max of the three */
  double pobj, dobj;         /* 1/2<x,Qx> + <c,x> + phi(x) and its dual counterpart */
  int64_t iters, restarts;
  double sigma, lambda_A, lambda_Q;
  double solve_seconds;      /* wall time of the last hprqp_solve (power method included) */
  double power_seconds;      /* part of it spent in the power method */
  int64_t kernel_launches;   /* kernels of this library launched by the last solve */
  int32_t status;
  /* tolerance ladder (Sec. 4 reports 1e-4, 1e-6 and 1e-8): the first stopping test at which
   * max(eta_p, eta_d, eta_gap) <= 1e-4 (resp. 1e-6), and the time to it (power method plus
   * device time from the first step to that test); 0 when not reached */
  int64_t iters_1e4, iters_1e6;
  double seconds_1e4, seconds_1e6;
  /* SpMV schedule picked at create: lanes per row of the Q, A and A^T passes and of the
   * factor pre-pass (0: the staged chunk form); 0 throughout from the batched solver */
  int32_t lanes_q, lanes_a, lanes_at, lanes_pre;
  int32_t tiled_terms;       /* factor terms whose one-vector products use shared-memory tiles */
} hprqp_kkt;

/* One stopping test of a solve (every check_every iterations, Sec. 4.1). */
typedef struct hprqp_check {
  int64_t iter, restarts;    /* iterations and restarts completed at the test */
  double sigma;              /* penalty parameter in use */
  double eta_p, eta_d, eta_gap, pobj, dobj;
  double R;                  /* the last R~ of eq. (2.12) evaluated */
  double seconds;            /* device time since the first inner step */
} hprqp_check;

/* Kernel kinds reported by hprqp_profile. */
enum {
  HPRQP_PROF_ZX = 0,         /* pending Halpern/restart update + eqs. (3.1)-(3.3), elementwise */
  HPRQP_PROF_PRE1 = 1,       /* B_f wbar_{1/2}, F_g wbar_{1/2} (factor terms of Q) */
  HPRQP_PROF_Q1 = 2,         /* Q wbar_{1/2} and v = what + sigma (Q w - Q wbar_{1/2}) */
  HPRQP_PROF_A1 = 3,         /* A v, Halpern on y, eq. (3.5) */
  HPRQP_PROF_AT = 4,         /* A^T ybar and wbar of eq. (3.3) */
  HPRQP_PROF_PRE2 = 5,       /* B_f wbar, F_g wbar */
  HPRQP_PROF_Q2 = 6,         /* Q wbar, R~ / stopping sums, controller */
  HPRQP_PROF_RPRE = 7,       /* restart: B_f d, F_g d */
  HPRQP_PROF_RESTART = 8,    /* restart: theta~ of eq. (3.11), Algorithm 5 */
  HPRQP_PROF_ATH = 9,        /* fused: A^T ybar, wbar, then the next Halpern update of w_Q, A^* y */
  HPRQP_PROF_PREW = 10,      /* fused: B_f w_Q, F_g w_Q of the new iterate */
  HPRQP_PROF_Q2H = 11,       /* fused: Q w_Q of the new iterate, the next step's Halpern update of
                                x and eqs. (3.1)-(3.3), controller */
  HPRQP_PROF_KINDS = 12
};

typedef struct hprqp_handle hprqp_handle;

/* Fills p with the defaults of Sec. 4.1 (alphas, tolerances) and the library defaults. */
void hprqp_default_params(hprqp_params* p);

/* Creates a solver for eq. (1.1).  n > 0 variables, m >= 0 rows.  A is CSR (m+1 row
 * pointers; may all be NULL when m == 0).  c, L, U have n entries; l, u have m.  L, U may
 * be NULL for phi = HPRQP_PHI_L1 (treated as -inf/+inf).  lambda >= 0 is the l1 weight.
 * All inputs are copied (host or device, detected per pointer); the caller keeps ownership
 * of its buffers and may free them after the call.  params may be NULL (defaults).
 * Builds A^T (and B^T for every FACTOR term) on the device.
 * Returns HPRQP_INVALID_ARG for inconsistent sizes, NaN, l > u, L > U, l or L = +INFINITY,
 * u or U = -INFINITY, non-monotone row pointers or out-of-range column indices; HPRQP_OOM / HPRQP_CUDA_ERROR on device failure.
 * On failure *h is set to NULL and nothing is leaked. */
hprqp_status hprqp_create(hprqp_handle** h, int64_t n, int64_t m, const hprqp_qop* Q,
                          const int32_t* A_rowptr, const int32_t* A_colidx, const double* A_vals,
                          const double* c, const double* l, const double* u, const double* L,
                          const double* U, int32_t phi, double lambda, const hprqp_params* params);

/* Sets the starting point u^{0,0} of Algorithm 4: x^0 = x0 (n), y^0 = y0 (m), w^0 = x0
 * (Q w* = Q x* at a solution, eq. (2.1)), z^0 = 0.  Either pointer may be NULL (zeros).
 * sigma0 > 0 replaces the initial penalty parameter; <= 0 keeps the Sec. 4.1 rule.
 * The warm start stays in effect for later solves until called again with NULLs. */
hprqp_status hprqp_set_warm_start(hprqp_handle* h, const double* x0, const double* y0, double sigma0);

/* Runs Algorithm 4 from the starting point until max(eta_p, eta_d, eta_gap) <= tol (tested
 * every check_every iterations), max_iter iterations (>= 1), or the time limit.  Includes
 * the power method for lambda_A, lambda_Q unless fixed in params.  Returns HPRQP_OK,
 * HPRQP_MAX_ITER, HPRQP_TIME_LIMIT or HPRQP_NUMERICAL_ERROR (or an error status). */
hprqp_status hprqp_solve(hprqp_handle* h, double tol, int64_t max_iter);

/* Copies the output bar iterate of Algorithm 4 (xbar: n, ybar: m, zbar: n, wbar_Q: n) into
 * caller buffers (host or device; any may be NULL) and fills kkt (may be NULL). */
hprqp_status hprqp_get(hprqp_handle* h, double* x, double* y, double* z, double* w, hprqp_kkt* kkt);

/* Applies one linear operator of problem (1.1) (Sec. 1) to a vector (for tests and
 * benchmarks): op 0: out = A in (in: n, out: m); 1: out = A^T in (in: m, out: n);
 * 2: out = Q in (n -> n).  in/out may be host or device pointers; with preconditioning they
 * are in the original variables. */
hprqp_status hprqp_apply(hprqp_handle* h, int32_t op, const double* in, double* out);

/* Runs `iters` (>= 1) inner steps of Algorithm 4 from the starting point, with lambda_A,
 * lambda_Q and sigma0 of the last hprqp_solve, as individual launches on the handle's stream
 * bracketed by CUDA events, and writes the mean duration (milliseconds) of each kernel kind
 * into ms[HPRQP_PROF_KINDS]: the step kinds over the plain steps (the steps with the R~ or the
 * stopping test carry extra sums; over all steps when none was plain), the restart kinds
 * over the steps that restarted, 0 for kinds the problem does not use.  The iterate is left in an unspecified state:
 * call hprqp_solve again before hprqp_get.  Requires a previous hprqp_solve. */
hprqp_status hprqp_profile(hprqp_handle* h, int32_t iters, double* ms);

/* Copies the records of the stopping tests of the last hprqp_solve (Algorithm 4 only; the
 * last 512 are kept), oldest first, into out (host memory, cap entries) and sets *count. */
hprqp_status hprqp_history(hprqp_handle* h, hprqp_check* out, int32_t cap, int32_t* count);

/* Allocation-free power method.  The paper has no counterpart to this entry point; it exists
 * for callers that cannot allocate device memory at the moment they need lambda_A: real-time
 * loops that must not allocate after start-up (an allocation may block), and processes whose
 * device memory is owned entirely by another allocator (a framework's pool that leaves nothing
 * for cudaMalloc).
 *
 * Computes lambda_A = safety * lambda_1(A A^*) exactly as hprqp_solve does (same start vector,
 * Rayleigh quotient and stopping rule: relative change <= tol, at most max_iter steps) and
 * writes it to *lambda_out (host pointer).  A (m x n) and its transpose A^T (n x m) are CSR
 * arrays in device memory; stream is a cudaStream_t (NULL: the legacy default stream).
 *
 * Nothing is allocated: the work vectors, partial sums and control scalars live in one
 * file-scope device array sized for m, n <= HPRQP_NOALLOC_MAX_DIM, which every GPU that loads
 * the library keeps until the process exits (about 3.2 MB).  Larger m or n return
 * HPRQP_INVALID_ARG.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress).  All calls share the array; calls that overlap on the GPU race with
 * each other.  The call synchronizes `stream` (it copies the row-pointer ends and the
 * convergence flag to the host), so it cannot be used on a stream that is being captured into a
 * CUDA graph.  It returns after the estimate has been copied to the host. */
#define HPRQP_NOALLOC_MAX_DIM 131072
hprqp_status hprqp_power_noalloc(int64_t m, int64_t n, const int32_t* A_rowptr, const int32_t* A_colidx,
                                 const double* A_vals, const int32_t* AT_rowptr, const int32_t* AT_colidx,
                                 const double* AT_vals, int64_t max_iter, double tol, double safety,
                                 void* stream, double* lambda_out);

/* Releases all device memory of the handle.  NULL is ignored. */
void hprqp_destroy(hprqp_handle* h);

/* Bookkeeping, with no counterpart in the paper: sets hprqp_params.wait_polls of the handle for
 * later solves (launch_mode 3: polls of one grid-barrier wait; 0 restores the default).  A solve
 * whose wait gave up returns HPRQP_TIMEOUT; every solve starts from a cleared barrier. */
hprqp_status hprqp_set_wait_polls(hprqp_handle* h, int32_t polls);

/* Bookkeeping, with no counterpart in the paper: the device memory the handle holds, by the
 * path it came from.  out[0], out[1]: allocations and bytes obtained through the allocator
 * hooks of hprqp_params (alloc/free); out[2], out[3]: allocations and bytes obtained with
 * cudaMalloc (when no hook is set).  Host pointer to 4 int64 values. */
hprqp_status hprqp_memory_stats(const hprqp_handle* h, int64_t* out);

/* Measurement utility with no counterpart in the paper: the issue rate of one arithmetic
 * operation on the current device, the roof that bounds this library's FP64 kernels on
 * GB300.  op: 0 FP64 FMA, 1 FP64 add, 2 FP64 multiply, 3 FP32 FMA (for comparison).
 * A full wave of 256-thread blocks (all resident at once) runs eight independent chains of
 * the operation per thread with the first `lanes` (1..32) lanes of each warp active.
 * Outputs (host pointers): *lanes_per_clk = thread operations per SM clock per SM (from the
 * blocks' clock64 spans); *sm_mhz = the SM clock during the run (clock64 cycles over the
 * CUDA-event duration); *ops_per_s = thread operations per second for the whole device.
 * sm_mhz and ops_per_s may be NULL.  Allocates and frees two small buffers; synchronizes
 * the device's legacy default stream.  HPRQP_INVALID_ARG for op or lanes out of range. */
hprqp_status hprqp_fp64_rate(int32_t op, int32_t lanes, double* lanes_per_clk, double* sm_mhz, double* ops_per_s);

/* ------------------------------------------------------------------------------------------
 * Batched solver: many independent instances of eq. (1.1), each run through Algorithm 4 with
 * its own sigma, restart and termination state.  Instances are bucketed by n, and each bucket
 * runs as one persistent kernel launch in which a thread block (64 to 512 threads, chosen per
 * bucket by an autotuner that times the candidates on the batch itself, as is a shared-memory
 * copy of the instance's dense factor) solves one instance at a time, taking the next from the
 * bucket's work queue (largest estimated cost first).  The launches of the buckets overlap on
 * internal streams forked from and joined back to the batch's stream.
 * Supported Q terms per instance: at most one DIAG, one DENSE_FACTOR (p <= 1024) and one CSR.
 * m <= HPRQP_BATCH_MAX_M rows per instance (the second Q product of a step and the theta
 * terms of eqs. (2.12), (3.11) use Q A^T and A Q A^T, formed once per solve).
 * ---------------------------------------------------------------------------------------- */
#define HPRQP_BATCH_MAX_M 32
#define HPRQP_BATCH_MAX_P 1024

typedef struct hprqp_problem {
  int64_t n, m;
  const hprqp_qop* Q;
  const int32_t* A_rowptr;   /* m+1 */
  const int32_t* A_colidx;
  const double* A_vals;
  const double *c, *l, *u, *L, *U;   /* as in hprqp_create; L, U may be NULL for PHI_L1 */
  int32_t phi;
  double lambda;
  const double* x0;          /* optional warm start (NULL: origin), w0 = x0 */
  const double* y0;
  double sigma0;             /* > 0: initial sigma; else the Sec. 4.1 rule */
  double lambda_A, lambda_Q; /* > 0: use as given; else the power method of Sec. 4.1 */
} hprqp_problem;

typedef struct hprqp_batch hprqp_batch;

/* Copies `count` (>= 1) problems (host or device pointers) to the device.  params: as for
 * hprqp_create (stream, alphas, periods, power method, autotune, batch_team; NULL = defaults).
 * The autotuner times each bucket's block size and F copy on a sample of the bucket at the first
 * solve.  Batched instances are solved without the Sec. 4.1 preconditioning (params.scaling
 * is ignored). */
hprqp_status hprqp_batch_create(hprqp_batch** b, int32_t count, const hprqp_problem* probs,
                                const hprqp_params* params);
/* Runs Algorithm 4 on every instance until its Sec. 4.1 stopping rule,
 * max(eta_p, eta_d, eta_gap) <= tol, holds or max_iter iterations have run.  Returns HPRQP_OK
 * when all converged, HPRQP_MAX_ITER when some did not, an error status otherwise. */
hprqp_status hprqp_batch_solve(hprqp_batch* b, double tol, int64_t max_iter);
/* The bar iterate (xbar, ybar, zbar) of instance i, the output of Algorithm 4, and its
 * stopping-rule values (Sec. 4.1); any output may be NULL; host or device. */
hprqp_status hprqp_batch_get(hprqp_batch* b, int32_t i, double* x, double* y, double* z, hprqp_kkt* kkt);
/* Bookkeeping, with no counterpart in the paper: the wall time (seconds) of the last
 * hprqp_batch_solve and the number of kernel launches in it; destroy (NULL is a no-op);
 * the message of the last failure on the batch ("" if none; b = NULL gives the last failure
 * of hprqp_batch_create in this thread). */
hprqp_status hprqp_batch_stats(hprqp_batch* b, double* seconds, int64_t* kernel_launches);
/* Bookkeeping, with no counterpart in the paper: the schedule the autotuner chose at the first
 * hprqp_batch_solve.  Instances are bucketed by n (largest first); for each of the 4 buckets,
 * out[5*k .. 5*k+4] = smallest n of the bucket, instances in it, threads per instance (the block
 * size, 64..512), 1 if a block keeps its instance's dense factor F in shared memory (else 0),
 * and that copy's capacity in doubles.  Host pointer to 20 int64. */
hprqp_status hprqp_batch_schedule(const hprqp_batch* b, int64_t* out);
void hprqp_batch_destroy(hprqp_batch* b);
const char* hprqp_batch_last_error(const hprqp_batch* b);

/* Bookkeeping, with no counterpart in the paper: the message of the last failure on this
 * handle ("" if none); h may be NULL for the last failure of hprqp_create in this thread. */
const char* hprqp_last_error(const hprqp_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* HPRQP_H */
