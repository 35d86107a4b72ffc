// Kernel argument block and launch helpers of the single-instance HPR-QP solver.
#pragma once
#include "core.cuh"

namespace hprqp {

struct Vec {
  // current iterate u = (y, w_Q, x) with the images Q w, A^* y; anchor u^{r,0}; bar iterate
  double *x, *w, *Qw, *ATy;
  double *x0, *w0, *Qw0, *ATy0;
  double *xb, *wb, *Qwb, *ATyb;
  double *wh, *Qwh, *v, *zb, *Qxb;
  double* xh;                 // what = 2 xbar - x of eq. (3.3), read by the Q wbar_{1/2} pass
  double *y, *y0, *yb;
  const double *c, *L, *U, *l, *u;
  double *t1, *t2;            // factor intermediates (2 * tlen each)
  double *pv, *pw, *ptmp;     // power method vectors
  const double* ain;          // apply input / output
  double* aout;
  // preconditioning (x = D xs, y = E ys): d, e and their reciprocals; null when not scaled
  const double *sd, *se, *isd, *ise;
};

// partial-sum regions (doubles); each kernel that reduces owns a region of gridDim.x rows
constexpr int kWL = 12;   // width of the end-of-iteration partials
constexpr int kW3 = 4;    // width of the y-step partials
constexpr int kWR = 5;    // width of the restart partials
constexpr int kWP = 2;    // width of the power-method partials

struct Args {
  int64_t n, m;
  int phi;
  Csr A, AT;
  QDev Q;
  Vec V;
  Ctrl* C;
  double* partL;
  double* part3;
  double* partR;
  double* partP;
  unsigned* counters;       // [0] end-of-iteration, [1] restart, [2] power
  int nbM;                  // blocks of the m-row kernel (rows of part3)
  CheckRec* hist;           // stopping-test records (kHistCap), or null
};

// Row-kernel kinds
// K_ATH, K_Q2H: the last two passes of a plain step whose successor starts with a Halpern step
// (no restart is possible after a plain step): K_ATH is K_AT followed by the Halpern update of
// (w_Q, A^* y); K_Q2H forms Q w of the new iterate directly (instead of Q wbar and the Halpern
// recurrence of the image) and runs the next step's elementwise pass (Halpern on x, eqs.
// (3.1)-(3.3)) in its epilogue, so that step needs no k_zx.
enum Kind { K_Q1 = 0, K_A1 = 1, K_AT = 2, K_Q2 = 3, K_APPLY_Q = 4, K_APPLY_A = 5, K_APPLY_AT = 6,
            K_POWER_Q = 7, K_POWER_A = 8, K_APPLY_AT_P = 9, K_ATH = 10, K_Q2H = 11 };
// kinds that run inside an inner step (they return once the solve is done)
__host__ __device__ constexpr bool step_kind(int k) { return k <= K_Q2 || k == K_ATH || k == K_Q2H; }

// Intermediate products formed before a Q pass (factor pre-pass, tiled factor kernels, QAP
// product), by source vector: 0 wbar_{1/2} (and xbar on stopping tests), 1 wbar, 2 the restart
// difference A^* ybar - A^* y^{r,0}, 3 the apply input, 4 the power-method vector, 5 w_Q (the
// new Halpern iterate, for K_Q2H).  Sources 0, 3 and 4 fill t1, the others t2.
enum PreSrc { PRE_WH = 0, PRE_WB = 1, PRE_RDIFF = 2, PRE_AIN = 3, PRE_PV = 4, PRE_W = 5 };
__host__ __device__ constexpr bool pre_into_t1(int which) { return which == PRE_WH || which == PRE_AIN || which == PRE_PV; }
// sources used by the inner step (idle once the solve is done)
__host__ __device__ constexpr bool pre_in_step(int which) { return which <= PRE_RDIFF || which == PRE_W; }

// Launch plan chosen at create time (lanes per row of each CSR pass, grid sizes).
struct Plan {
  int gQ = 1, gA = 1, gAT = 1, gPre = 32;   // lanes per row (0: staged chunk form)
  int gridN = 0, gridM = 0, gridE = 0, gridPre = 0;   // blocks of the n-row, m-row, elementwise, pre kernels
  // blocks of the plain (non-reducing) step variants: one full wave at the occupancy of each
  // kernel; the reducing variants keep gridN/gridM/gridE, which size the partial-sum regions
  int wZX = 0, wQ1 = 0, wA1 = 0, wAT = 0, wQ2 = 0, wATH = 0, wQ2H = 0;
  // fixed-schedule graph: plain steps end with K_ATH + K_Q2H, which run the next step's
  // elementwise pass (requires Q and A)
  int fuse = 0;
  int gridP = 0;   // blocks of the persistent (cooperative) solver
  int gridT = 0;   // blocks of the tiled B^T t kernel
  // programmatic dependent launch between consecutive kernels of a step (each kernel waits for
  // its predecessor with griddepcontrol.wait, so only its launch overlaps the predecessor's end)
  int pdl = 0;
};

// Halpern weights 1/(i+2), (i+1)/(i+2) of the step after the current one (Algorithm 4; i the
// inner counter t, or k with halpern_total), evaluated before the controller advances t and k.
// The controller and the fused passes use this one expression, so their weights agree bit for bit.
__host__ __device__ inline void halpern_weights(const Ctrl& C, double& ha, double& hb) {
  const double i = C.halpern_total ? (double)C.k : (double)C.t;
  ha = 1.0 / (i + 2.0);
  hb = (i + 1.0) / (i + 2.0);
}

// sigma and the scalars derived from it (host and device use the same arithmetic)
__host__ __device__ inline void set_sigma(Ctrl& C, double sigma) {
  C.sigma = sigma;
  C.inv_sigma = 1.0 / sigma;
  const double d = 1.0 + sigma * C.lamQ;
  C.c1 = sigma * C.lamQ / d;
  C.c2 = 1.0 / d;
  C.s = sigma / d;
  C.slA = sigma * C.lamA;
  C.inv_slA = C.slA > 0.0 ? 1.0 / C.slA : 0.0;
  C.tau = sigma * C.lambda;
}

// host-side launchers (solver.cu)
// One inner step; var: 0 plain, 1 with the R~ test, 2 with the stopping test, 3 decided on the
// device at run time.  ev (optional) receives CUDA events around each kernel kind.
cudaError_t launch_step_var(const Args& a, const Plan& p, cudaStream_t s, int var, cudaEvent_t (*ev)[2] = nullptr);
cudaError_t launch_iteration(const Args& a, const Plan& p, cudaStream_t s, cudaEvent_t (*ev)[2] = nullptr);
// One inner step as the fixed-schedule graph runs it: k1 false when the previous step's K_Q2H
// ran this step's elementwise pass; fuse_next >= 0 (plain steps, p.fuse): end with K_ATH and
// K_Q2H for a next step of that variant.
cudaError_t launch_step_fused(const Args& a, const Plan& p, cudaStream_t s, int var, bool k1, int fuse_next,
                              cudaEvent_t (*ev)[2] = nullptr);
cudaError_t launch_restart(const Args& a, const Plan& p, cudaStream_t s, cudaEvent_t (*ev)[2] = nullptr);
cudaError_t build_conditional_graph(const Args& a, const Plan& p, cudaStream_t s, cudaStream_t s2, int steps,
                                    cudaGraph_t* out);
// Graph of L steps whose variants are fixed by position (R~ test every re, stopping test
// every ce steps; L a multiple of both), one SWITCH node after each R~ test for the restart.
// *kernels (optional) receives the number of kernels one launch runs when no restart happens.
cudaError_t build_fixed_graph(const Args& a, const Plan& p, cudaStream_t s, cudaStream_t s2, int L, int re, int ce,
                              cudaGraph_t* out, int* kernels = nullptr);
int kernels_per_step(const Args& a);
int kernels_per_restart(const Args& a);
int kernels_per_iteration(const Args& a);
cudaError_t launch_apply(const Args& a, const Plan& p, int op, cudaStream_t s);
cudaError_t launch_power_iter(const Args& a, const Plan& p, int which, int i, cudaStream_t s);
int kernels_per_power_iter(const Args& a, int which);
cudaError_t launch_power_init(const Args& a, const Plan& p, int which, cudaStream_t s);
cudaError_t launch_zbar(const Args& a, const Plan& p, cudaStream_t s);
cudaError_t launch_spmv_probe(const Csr& M, int G, int grid, const double* x, double* y, cudaStream_t s);
cudaError_t launch_pre_probe(const Args& a, int G, int grid, cudaStream_t s);
// shared-memory-tiled factor products (tiled.cu): t = B_f x, then (which != 2) u = B_f^T t,
// for every tiled factor term; *launched receives the number of kernels
cudaError_t tiled_setup();
int tiled_tbt_grid(int64_t n, int sms);
cudaError_t launch_tiled(const Args& a, const Plan& p, int which, int tt, cudaStream_t s, int* launched);
// v[i] *= s[i] for i < n
cudaError_t launch_vmul(double* v, const double* s, int64_t n, cudaStream_t st);
// out[i] = v[i] * s[i] for i < n
cudaError_t launch_vmul_to(double* out, const double* v, const double* s, int64_t n, cudaStream_t st);
// Persistent solver (persist.cu): co-resident blocks of its kernel on `sms` SMs, and one
// cooperative launch running at most `steps` inner steps (bar: 2 zeroed words; err: flag; spin:
// polls of one barrier wait, 0 for the default of about a second).
int persist_max_blocks(int sms);
cudaError_t launch_persist(const Args& a, const Plan& p, int grid, long long steps, unsigned* bar, int* err,
                           unsigned spin, cudaStream_t s);
// Primal HPR methods of Appendix A (primal.cu): the elementwise steps and the stopping rule
cudaError_t primal_rows(const double* Ax, const double* y, const double* l, const double* u, double sigma, int64_t m,
                        double* sb, double* yb, double* w, cudaStream_t s);
cudaError_t primal_vt(const double* v, const double* Qv, const double* x, const double* t, double lamQ, double sigma,
                      int64_t n, double* vb, double* tb, cudaStream_t s);
cudaError_t primal_x(const double* x, const double* Qv, const double* c, const double* ATw, const double* vb,
                     const double* tb, const double* L, const double* U, int phi, double lambda, double sigma,
                     double tau, int two, int64_t n, double* xb, double* zb, cudaStream_t s);
cudaError_t primal_halpern(double* const* u, const double* const* u0, const double* const* ub, int count, double a,
                           double b, int64_t len, cudaStream_t s);
int primal_eta_blocks(int64_t len);
cudaError_t primal_eta(const double* xb, const double* Qxb, const double* ATyb, const double* zb, const double* Axb,
                       const double* yb, const Args& a, double b_inf, double c_inf, double lambda, double* part_n,
                       double* part_m, double* out, cudaStream_t s);
// The QAP term's product(s) before a pass that needs them (which as for k_pre; tt: 0 one
// vector, 1 or 2 also x-bar for the stopping test); no-op without a QAP term.
cudaError_t launch_qap(const Args& a, const Plan& p, int which, int tt, cudaStream_t s);
// qap.cu: out = vec(Ahat X Bhat - S X - X T) for x = vec(X) (two kernels), and the K-range
// split that keeps about two blocks per SM busy for a d x d product
constexpr int kQapMaxSplits = 8;
cudaError_t qap_apply(const QDev& Q, const double* x, double* out, int splits, cudaStream_t s);
int qap_splits(int64_t d, int sms);
// Records the device time stamp of the start of the iteration (tolerance ladder).
cudaError_t launch_stamp(const Args& a, cudaStream_t s);
// Fills the plain-variant grids of p from the occupancy of those kernels (after gQ, gA, gAT).
cudaError_t plan_plain_grids(const Args& a, Plan& p, int sms);

}  // namespace hprqp
