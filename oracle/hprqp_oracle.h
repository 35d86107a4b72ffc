/* HPR-QP reference oracle: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 C implementation of HPR-QP (Algorithm 4 with the
 * SigmaUpdate of Algorithm 5) used to check the CUDA library.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header or constant with the CUDA library.
 *
 * Problem (Sec. 1, eq. (1.1)):  min 1/2<x,Qx> + <c,x> + phi(x)   s.t.  Ax in K = [l,u]
 * with phi the indicator of C = [L,U] (eq. (1.2)), lam*||x||_1, or both.
 */
#ifndef HPRQP_ORACLE_H
#define HPRQP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_Q_DIAG = 1, ORC_Q_CSR = 2, ORC_Q_DIA = 3, ORC_Q_FACTOR = 4, ORC_Q_DENSE = 5, ORC_Q_QAP = 6 };
enum { ORC_PHI_BOX = 0, ORC_PHI_L1 = 1, ORC_PHI_L1_BOX = 2 };
enum { ORC_CONVERGED = 0, ORC_MAX_ITER = 1, ORC_NUMERICAL = 3, ORC_INVALID = 4 };

/* One additive term of Q (Q is the sum of its terms; no terms means Q = 0). */
typedef struct {
  int32_t kind;
  int64_t p;                 /* FACTOR / DENSE: rows of B or F */
  const int32_t* rowptr;     /* CSR (n x n) or FACTOR B (p x n) */
  const int32_t* colidx;
  const double* vals;
  int32_t ndiag;             /* DIA: symmetric band, offsets >= 0 */
  const int32_t* offsets;
  const double* diags;       /* DIA: ndiag x n, diags[k*n+i] = Q[i][i+off_k] */
  const double* dense;       /* DIAG: n entries; DENSE: F row-major p x n; QAP: the symmetric
                                d x d matrices Ahat, Bhat, S, T one after another (p = d,
                                n = d^2), Q vec(X) = vec(Ahat X Bhat - S X - X T) with
                                vec(X)[i + j d] = X[i][j] (Sec. 4.5) */
} orc_qterm;

typedef struct {
  int64_t n, m;
  int32_t nq;
  const orc_qterm* q;
  const int32_t* A_rowptr;   /* m+1 */
  const int32_t* A_colidx;
  const double* A_vals;
  const double *c, *l, *u, *L, *U;
  int32_t phi;
  double lambda;
} orc_problem;

typedef struct {
  double tol;
  int64_t max_iter;
  int64_t check_every;       /* termination test period (iterations) */
  int64_t restart_every;     /* restart test period (iterations)     */
  double alpha1, alpha2, alpha3, alpha3_tight, ratio_tight;
  double lambda_A, lambda_Q; /* <= 0: estimate with the power method */
  double sigma0;             /* <= 0: ||b||/||c|| rule of Sec. 4.1   */
  int64_t power_max_iter;
  double power_tol, power_safety;
  int32_t halpern_total;     /* 1: Halpern weight from the total counter k */
  int32_t sigma_golden;      /* 1: golden-section search instead of the exact argmin */
  int32_t restart_off;       /* 1: never restart (plain Algorithm 3) */
  int32_t sigma_fixed;       /* 1: keep sigma0 at restarts */
  int32_t scaling;           /* 1: Ruiz + Pock-Chambolle preconditioning of Sec. 4.1 when Q is
                                explicit (DIAG/CSR/DIA terms only) and phi is the box indicator */
  int32_t method;            /* 0: dual HPR-QP (Algorithm 4); 1: primal HPR on (1.3)
                                (Algorithm 6); 2: primal HPR on (1.4) (Algorithm 7).  The primal
                                methods run as printed: fixed sigma (sigma0), no restarts, and
                                without preconditioning */
  const double* x0;          /* optional warm start (n); w0 = x0 */
  const double* y0;          /* optional warm start (m) */
  /* optional per-iteration trace (first trace_len iterations), any may be NULL */
  int64_t trace_len;
  double* trace_x;           /* trace_len x n : xbar */
  double* trace_y;           /* trace_len x m : ybar */
  double* trace_R;           /* trace_len : R~ (NaN where not evaluated) */
  double* trace_sigma;       /* trace_len : sigma used in the iteration */
  int32_t* trace_restart;    /* trace_len : 1 if the iteration ended with a restart */
  double* trace_w;           /* trace_len x n : wbar_Q */
} orc_params;

typedef struct {
  double eta_p, eta_d, eta_gap, pobj, dobj;
  int64_t iters, restarts;
  double sigma, lambda_A, lambda_Q;
  int32_t status;
  int64_t iters_1e4, iters_1e6;  /* first stopping test with max(eta) <= 1e-4 / 1e-6 (0: none) */
} orc_result;

void orc_default_params(orc_params* p);
/* Sec. 4.1 preconditioning: 10 Ruiz passes, then Pock-Chambolle with alpha = 1, on
 * K = [Q A^T; A 0]; writes the column scaling d (n) and row scaling e (m) of
 * x = D xs, y = E ys.  Returns 0 (d = e = 1) when the problem is not eligible. */
int orc_scaling(const orc_problem* P, double* d, double* e);

/* Algorithm 4.  x, y, z, w receive the final bar iterate (any may be NULL). */
int orc_solve(const orc_problem* P, const orc_params* prm, orc_result* res,
              double* x, double* y, double* z, double* w);

/* building blocks exposed for the pins */
void orc_qmul(const orc_problem* P, const double* v, double* out);
void orc_amul(const orc_problem* P, const double* v, double* out);
void orc_atmul(const orc_problem* P, const double* v, double* out);
double orc_power_A(const orc_problem* P, int64_t max_iter, double tol, double safety);
double orc_power_Q(const orc_problem* P, int64_t max_iter, double tol, double safety);
double orc_sigma_argmin(double t1, double t2, double t3, double lamQ, int golden);
double orc_sigma_update(double th1, double th2, double th3, double lamQ, double ratio, double sigma_r,
                        int golden);
double orc_mnorm2(const orc_problem* P, double sigma, double lamA, double lamQ,
                  const double* dy, const double* dw, const double* dx);
void orc_eta(const orc_problem* P, const double* xb, const double* yb, const double* zb,
             double* eta3, double* pobj, double* dobj);
/* one fixed-sigma inner step of Algorithm 3 from (y, w, x): fills the bar iterate */
void orc_step(const orc_problem* P, double sigma, double lamA, double lamQ,
              const double* y, const double* w, const double* x,
              double* yb, double* wb, double* zb, double* xb, double* wh);

#ifdef __cplusplus
}
#endif
#endif
