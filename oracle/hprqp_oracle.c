/* HPR-QP reference oracle: TEST INFRASTRUCTURE ONLY (see hprqp_oracle.h).
 *
 * Plain single-threaded FP64.  Every operator product is formed afresh from the stored
 * matrices in the order the paper writes the update; nothing is fused, cached or
 * reordered.  Compile with -ffp-contract=off so that no multiply-add is fused.
 *
 * Sources (arXiv 2507.02470):
 *   Algorithm 4 (HPR-QP), Sec. 3, with the subproblem solutions of Sec. 3.1:
 *     eq. (3.1) z-update, eq. (3.2) x-update, eq. (3.3) w-updates (shadow sequence of
 *     Prop. 3.1), eq. (3.4) S_y = lam_A I - A A^*, eq. (3.5) y-update;
 *   Sec. 3.2 restart criteria (3.6)-(3.8) on R~ = ||u - ubar||_M with M of eq. (2.12);
 *   Sec. 3.3 sigma update: eqs. (3.10)-(3.12) and Algorithm 5 (SigmaUpdate);
 *   Sec. 4.1 parameter settings (power method, sigma0, alphas) and the stopping rule.
 */
#include "hprqp_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ small vector ops */
static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
  return s;
}
static double nrm2(const double* a, int64_t n) { return sqrt(dot(a, a, n)); }
static double nrminf(const double* a, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; i++) s = fmax(s, fabs(a[i]));
  return s;
}
static double* vnew(int64_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* ------------------------------------------------------------------ linear operators */
/* Q v: sum of the terms (Sec. 1: Q need not be an explicit matrix). */
void orc_qmul(const orc_problem* P, const double* v, double* out) {
  int64_t n = P->n;
  for (int64_t i = 0; i < n; i++) out[i] = 0.0;
  for (int32_t t = 0; t < P->nq; t++) {
    const orc_qterm* q = &P->q[t];
    if (q->kind == ORC_Q_DIAG) {
      for (int64_t i = 0; i < n; i++) out[i] += q->dense[i] * v[i];
    } else if (q->kind == ORC_Q_CSR) {
      for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t k = q->rowptr[i]; k < q->rowptr[i + 1]; k++) s += q->vals[k] * v[q->colidx[k]];
        out[i] += s;
      }
    } else if (q->kind == ORC_Q_DIA) {
      /* symmetric band: entry (i, i+o) = (i+o, i) = diags[k][i] */
      for (int32_t k = 0; k < q->ndiag; k++) {
        int64_t o = q->offsets[k];
        const double* d = q->diags + (int64_t)k * n;
        for (int64_t i = 0; i + o < n; i++) {
          out[i] += d[i] * v[i + o];
          if (o != 0) out[i + o] += d[i] * v[i];
        }
      }
    } else if (q->kind == ORC_Q_FACTOR) {
      /* B^T (B v) */
      double* t1 = vnew(q->p);
      for (int64_t r = 0; r < q->p; r++) {
        double s = 0.0;
        for (int32_t k = q->rowptr[r]; k < q->rowptr[r + 1]; k++) s += q->vals[k] * v[q->colidx[k]];
        t1[r] = s;
      }
      for (int64_t r = 0; r < q->p; r++)
        for (int32_t k = q->rowptr[r]; k < q->rowptr[r + 1]; k++) out[q->colidx[k]] += q->vals[k] * t1[r];
      free(t1);
    } else if (q->kind == ORC_Q_QAP) {
      /* Sec. 4.5: Q vec(X) = vec(Ahat X Bhat - S X - X T), all four d x d and symmetric */
      const int64_t d = q->p;
      const double *Ah = q->dense, *Bh = q->dense + d * d, *S = q->dense + 2 * d * d, *T = q->dense + 3 * d * d;
      double* AX = vnew(d * d);
      for (int64_t i = 0; i < d; i++)
        for (int64_t j = 0; j < d; j++) {
          double s = 0.0;
          for (int64_t k = 0; k < d; k++) s += Ah[i * d + k] * v[k + j * d];
          AX[i + j * d] = s;
        }
      for (int64_t i = 0; i < d; i++)
        for (int64_t j = 0; j < d; j++) {
          double s = 0.0;
          for (int64_t k = 0; k < d; k++) s += AX[i + k * d] * Bh[k * d + j];
          for (int64_t k = 0; k < d; k++) s -= S[i * d + k] * v[k + j * d];
          for (int64_t k = 0; k < d; k++) s -= v[i + k * d] * T[k * d + j];
          out[i + j * d] += s;
        }
      free(AX);
    } else if (q->kind == ORC_Q_DENSE) {
      /* F^T (F v), F row-major p x n */
      double* t1 = vnew(q->p);
      for (int64_t r = 0; r < q->p; r++) t1[r] = dot(q->dense + r * n, v, n);
      for (int64_t r = 0; r < q->p; r++)
        for (int64_t j = 0; j < n; j++) out[j] += q->dense[r * n + j] * t1[r];
      free(t1);
    }
  }
}

/* A v: the linear operator of the constraint Ax in K (Sec. 1), stored as CSR. */
void orc_amul(const orc_problem* P, const double* v, double* out) {
  for (int64_t i = 0; i < P->m; i++) {
    double s = 0.0;
    for (int32_t k = P->A_rowptr[i]; k < P->A_rowptr[i + 1]; k++) s += P->A_vals[k] * v[P->A_colidx[k]];
    out[i] = s;
  }
}

/* A^* y: the adjoint (transpose) of A, formed from the same CSR arrays row by row. */
void orc_atmul(const orc_problem* P, const double* v, double* out) {
  for (int64_t j = 0; j < P->n; j++) out[j] = 0.0;
  for (int64_t i = 0; i < P->m; i++)
    for (int32_t k = P->A_rowptr[i]; k < P->A_rowptr[i + 1]; k++) out[P->A_colidx[k]] += P->A_vals[k] * v[i];
}

/* ------------------------------------------------------------------ projections / prox */
static double clampd(double v, double lo, double hi) { return fmin(fmax(v, lo), hi); }

/* Prox_{sigma phi}(r) for phi = delta_C, lam||.||_1, or both (separable, Sec. 1). */
static double prox_phi(const orc_problem* P, int64_t j, double r, double sigma) {
  if (P->phi == ORC_PHI_BOX) return clampd(r, P->L[j], P->U[j]);
  double tau = sigma * P->lambda;
  double s = r - clampd(r, -tau, tau); /* soft threshold */
  if (P->phi == ORC_PHI_L1) return s;
  return clampd(s, P->L[j], P->U[j]);
}

/* phi(x) (x is feasible for the box by construction) */
static double phi_val(const orc_problem* P, const double* x) {
  if (P->phi == ORC_PHI_BOX) return 0.0;
  double s = 0.0;
  for (int64_t j = 0; j < P->n; j++) s += fabs(x[j]);
  return P->lambda * s;
}

/* a*b with the convention 0 * inf = 0 (a bound that carries no multiplier) */
static double mul0(double a, double b) { return (a == 0.0) ? 0.0 : a * b; }

/* delta*_K(-y) = sup_{s in K} <-y, s> = -sum_i [ l_i max(y_i,0) + u_i min(y_i,0) ] */
static double support_K(const orc_problem* P, const double* y) {
  double s = 0.0;
  for (int64_t i = 0; i < P->m; i++) s += mul0(fmax(y[i], 0.0), P->l[i]) + mul0(fmin(y[i], 0.0), P->u[i]);
  return -s;
}

/* phi*(-z) */
static double conj_phi(const orc_problem* P, const double* z) {
  double s = 0.0;
  if (P->phi == ORC_PHI_BOX) {
    for (int64_t j = 0; j < P->n; j++) s += mul0(fmax(z[j], 0.0), P->L[j]) + mul0(fmin(z[j], 0.0), P->U[j]);
    return -s;
  }
  if (P->phi == ORC_PHI_L1) return 0.0; /* indicator of [-lam, lam]^n, z bar lies inside */
  /* lam|x| + delta_[L,U]: per coordinate sup_{x in [L,U]} (-z x - lam |x|), a concave
     piecewise-linear function: the sup is at a finite end point or at 0 when z lies in the
     domain, i.e. z <= lam if L = -inf and z >= -lam if U = +inf.  zbar is a subgradient of
     phi at xbar (eq. (3.1)), so it lies there in exact arithmetic; (xbar - r_z)/sigma can
     cross the edge by rounding, so on an infinite side a z within 64 ulps of the edge
     (relative to max(1, lam)) is taken on the edge (as the pure l1 case above, whose
     conjugate is 0 on [-lam, lam], does).  A z further out is outside the domain: the
     conjugate is +inf. */
  const double edge = 64.0 * DBL_EPSILON * fmax(1.0, P->lambda);
  for (int64_t j = 0; j < P->n; j++) {
    double zj = z[j], Lj = P->L[j], Uj = P->U[j], lam = P->lambda, best = -INFINITY;
    if (!isfinite(Lj) && zj > lam) {
      if (zj - lam > edge) return INFINITY;
      zj = lam;
    }
    if (!isfinite(Uj) && zj < -lam) {
      if (-lam - zj > edge) return INFINITY;
      zj = -lam;
    }
    if (isfinite(Lj)) best = fmax(best, -zj * Lj - lam * fabs(Lj));
    if (isfinite(Uj)) best = fmax(best, -zj * Uj - lam * fabs(Uj));
    if (Lj <= 0.0 && Uj >= 0.0) best = fmax(best, 0.0);
    s += best;
  }
  return s;
}

/* ------------------------------------------------------------------ stopping rule (Sec. 4.1) */
void orc_eta(const orc_problem* P, const double* xb, const double* yb, const double* zb,
             double* eta3, double* pobj, double* dobj) {
  int64_t n = P->n, m = P->m;
  double* Ax = vnew(m);
  double* Qx = vnew(n);
  double* Aty = vnew(n);
  orc_amul(P, xb, Ax);
  orc_qmul(P, xb, Qx);
  orc_atmul(P, yb, Aty);
  /* eta_p = ||Ax - Pi_K(Ax)||_inf / (1 + max(||b||_inf, ||Ax||_inf)), b = max(|l|,|u|), inf -> 0 */
  double rp = 0.0, bnorm = 0.0;
  for (int64_t i = 0; i < m; i++) {
    rp = fmax(rp, fabs(Ax[i] - clampd(Ax[i], P->l[i], P->u[i])));
    double bl = isfinite(P->l[i]) ? fabs(P->l[i]) : 0.0;
    double bu = isfinite(P->u[i]) ? fabs(P->u[i]) : 0.0;
    bnorm = fmax(bnorm, fmax(bl, bu));
  }
  double eta_p = rp / (1.0 + fmax(bnorm, nrminf(Ax, m)));
  /* eta_d = ||-Qx + A^*y + z - c||_inf / (1 + max(||c||_inf, ||A^*y||_inf, ||Qx||_inf)) */
  double rd = 0.0;
  for (int64_t j = 0; j < n; j++) rd = fmax(rd, fabs(-Qx[j] + Aty[j] + zb[j] - P->c[j]));
  double eta_d = rd / (1.0 + fmax(nrminf(P->c, n), fmax(nrminf(Aty, n), nrminf(Qx, n))));
  /* eta_gap with primal value P and dual value D */
  double xQx = dot(xb, Qx, n);
  double pv = 0.5 * xQx + dot(P->c, xb, n) + phi_val(P, xb);
  double dv = -0.5 * xQx - support_K(P, yb) - conj_phi(P, zb);
  double eta_g = fabs(pv - dv) / (1.0 + fmax(fabs(pv), fabs(dv)));
  eta3[0] = eta_p;
  eta3[1] = eta_d;
  eta3[2] = eta_g;
  if (pobj) *pobj = pv;
  if (dobj) *dobj = dv;
  free(Ax);
  free(Qx);
  free(Aty);
}

/* ------------------------------------------------------------------ power method (Sec. 4.1) */
/* deterministic start vector: 0.5 + (hash(i) mod 2^32) / 2^32, exactly representable */
static double start_entry(int64_t i) {
  uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
  return 0.5 + (double)h / 4294967296.0;
}

static double power_generic(const orc_problem* P, int which, int64_t dim, int64_t max_iter, double tol,
                            double safety) {
  if (dim == 0) return 0.0;
  double* v = vnew(dim);
  double* w = vnew(dim);
  double* tmp = vnew(P->n > P->m ? P->n : P->m);
  for (int64_t i = 0; i < dim; i++) v[i] = start_entry(i);
  double nv = nrm2(v, dim);
  for (int64_t i = 0; i < dim; i++) v[i] /= nv;
  double lam = 0.0;
  for (int64_t it = 0; it < max_iter; it++) {
    if (which == 0) { /* A A^* on R^m */
      orc_atmul(P, v, tmp);
      orc_amul(P, tmp, w);
    } else {
      orc_qmul(P, v, w);
    }
    double lnew = dot(v, w, dim); /* Rayleigh quotient, ||v|| = 1 */
    double nw = nrm2(w, dim);
    if (nw == 0.0) { lam = 0.0; break; }
    for (int64_t i = 0; i < dim; i++) v[i] = w[i] / nw;
    int done = (it > 0) && fabs(lnew - lam) <= tol * fabs(lnew);
    lam = lnew;
    if (done) break;
  }
  free(v);
  free(w);
  free(tmp);
  return safety * lam;
}

double orc_power_A(const orc_problem* P, int64_t max_iter, double tol, double safety) {
  return power_generic(P, 0, P->m, max_iter, tol, safety);
}
double orc_power_Q(const orc_problem* P, int64_t max_iter, double tol, double safety) {
  if (P->nq == 0) return 0.0;
  return power_generic(P, 1, P->n, max_iter, tol, safety);
}

/* ------------------------------------------------------------------ sigma subproblem (eq. 3.12) */
static double fsig(double s, double t1, double t2, double t3, double lq) {
  return t1 * s + t2 / s + s * s * t3 / (1.0 + lq * s);
}
static double dfsig(double s, double t1, double t2, double t3, double lq) {
  double d = 1.0 + lq * s;
  return t1 - t2 / (s * s) + t3 * s * (2.0 + lq * s) / (d * d);
}

/* argmin_{s>0} t1 s + t2/s + s^2 t3/(1+lq s), t1, t2 > 0, t3 >= 0.  f is strictly convex;
 * since 0 <= d/ds[s^2/(1+lq s)] < 1/lq the minimiser lies in
 * [sqrt(t2/(t1 + t3/lq)), sqrt(t2/t1)].  exact: bisection on the monotone f';
 * golden: golden-section search on log s (f is convex in log s as well). */
double orc_sigma_argmin(double t1, double t2, double t3, double lq, int golden) {
  double hi = sqrt(t2 / t1);
  if (t3 <= 0.0 || lq <= 0.0) return hi;
  double lo = sqrt(t2 / (t1 + t3 / lq));
  if (!golden) {
    for (int it = 0; it < 200 && (hi - lo) > 4.0e-16 * hi; it++) {
      double mid = 0.5 * (lo + hi);
      if (dfsig(mid, t1, t2, t3, lq) > 0.0) hi = mid;
      else lo = mid;
    }
    return 0.5 * (lo + hi);
  }
  const double gr = 0.6180339887498949;
  double a = log(lo), b = log(hi);
  double c1 = b - gr * (b - a), c2 = a + gr * (b - a);
  double f1 = fsig(exp(c1), t1, t2, t3, lq), f2 = fsig(exp(c2), t1, t2, t3, lq);
  for (int it = 0; it < 200 && (b - a) > 1e-12; it++) {
    if (f1 < f2) {
      b = c2; c2 = c1; f2 = f1;
      c1 = b - gr * (b - a);
      f1 = fsig(exp(c1), t1, t2, t3, lq);
    } else {
      a = c1; c1 = c2; f1 = f2;
      c2 = a + gr * (b - a);
      f2 = fsig(exp(c2), t1, t2, t3, lq);
    }
  }
  return exp(0.5 * (a + b));
}

/* Algorithm 5 after the theta~ are formed: floor theta~_1, theta~_2 at 1e-12, minimise
 * eq. (3.12), then smooth in log sigma with beta = exp(-R~_{r,tau_r-1} / R~_{0,tau_0-1})
 * (``ratio`` is that quotient). */
double orc_sigma_update(double th1, double th2, double th3, double lamQ, double ratio, double sigma_r,
                        int golden) {
  th1 = fmax(th1, 1e-12);
  th2 = fmax(th2, 1e-12);
  double snew = orc_sigma_argmin(th1, th2, th3, lamQ, golden);
  double beta = exp(-ratio);
  return exp(beta * log(snew) + (1.0 - beta) * log(sigma_r));
}

/* ------------------------------------------------------------------ M-norm (eq. 2.12) */
/* ||(dy, dw, dz, dx)||_M^2 with T1 = S + S_sGS, S_y = lam_A I - AA^*, S_w = Q(lam_Q I - Q):
 *   sigma*th1 + th2/sigma + sigma^2 th3/(1+sigma lam_Q) + 2<dx, A^*dy - Q dw>,
 *   th1 = lam_A||dy||^2 + lam_Q<dw,Q dw> - 2<Q dw, A^*dy>, th2 = ||dx||^2,
 *   th3 = <A^*dy, Q A^*dy>; the z block of M is zero. */
double orc_mnorm2(const orc_problem* P, double sigma, double lamA, double lamQ, const double* dy,
                  const double* dw, const double* dx) {
  int64_t n = P->n, m = P->m;
  double* Qdw = vnew(n);
  double* Atdy = vnew(n);
  double* QAtdy = vnew(n);
  orc_qmul(P, dw, Qdw);
  orc_atmul(P, dy, Atdy);
  orc_qmul(P, Atdy, QAtdy);
  double th1 = lamA * dot(dy, dy, m) + lamQ * dot(dw, Qdw, n) - 2.0 * dot(Qdw, Atdy, n);
  double th2 = dot(dx, dx, n);
  double th3 = dot(Atdy, QAtdy, n);
  double cross = 0.0;
  for (int64_t j = 0; j < n; j++) cross += dx[j] * (Atdy[j] - Qdw[j]);
  free(Qdw);
  free(Atdy);
  free(QAtdy);
  return sigma * th1 + th2 / sigma + sigma * sigma * th3 / (1.0 + sigma * lamQ) + 2.0 * cross;
}

/* ------------------------------------------------------------------ one inner step (Sec. 3.1) */
void orc_step(const orc_problem* P, double sigma, double lamA, double lamQ, const double* y,
              const double* w, const double* x, double* yb, double* wb, double* zb, double* xb,
              double* wh) {
  int64_t n = P->n, m = P->m;
  double* Qw = vnew(n);
  double* Aty = vnew(n);
  double* Qwh = vnew(n);
  double* v = vnew(n);
  double* ry = vnew(m);
  double* Atdy = vnew(n);
  double* dy = vnew(m);
  orc_qmul(P, w, Qw);
  orc_atmul(P, y, Aty);
  for (int64_t j = 0; j < n; j++) {
    /* eq. (3.1)-(3.2): r_z = x + sigma(-Q w + A^* y - c), xbar = Prox_{sigma phi}(r_z),
       zbar = (xbar - r_z)/sigma */
    double rz = x[j] + sigma * (-Qw[j] + Aty[j] - P->c[j]);
    xb[j] = prox_phi(P, j, rz, sigma);
    zb[j] = (xb[j] - rz) / sigma;
    /* eq. (3.3): what = 2 xbar - x, wbar_{1/2} = (sigma lam_Q w + what)/(1 + sigma lam_Q) */
    double xh = 2.0 * xb[j] - x[j];
    wh[j] = (sigma * lamQ * w[j] + xh) / (1.0 + sigma * lamQ);
  }
  orc_qmul(P, wh, Qwh);
  /* eq. (3.5): r_y = A(what + sigma(Q w - Q wbar_{1/2})) - sigma lam_A y,
     ybar = (Pi_K(r_y) - r_y)/(sigma lam_A) */
  for (int64_t j = 0; j < n; j++) v[j] = (2.0 * xb[j] - x[j]) + sigma * (Qw[j] - Qwh[j]);
  orc_amul(P, v, ry);
  for (int64_t i = 0; i < m; i++) {
    ry[i] = ry[i] - sigma * lamA * y[i];
    yb[i] = (clampd(ry[i], P->l[i], P->u[i]) - ry[i]) / (sigma * lamA);
    dy[i] = yb[i] - y[i];
  }
  /* eq. (3.3): wbar = wbar_{1/2} + sigma/(1 + sigma lam_Q) A^*(ybar - y) */
  orc_atmul(P, dy, Atdy);
  for (int64_t j = 0; j < n; j++) wb[j] = wh[j] + sigma / (1.0 + sigma * lamQ) * Atdy[j];
  free(Qw);
  free(Aty);
  free(Qwh);
  free(v);
  free(ry);
  free(Atdy);
  free(dy);
}

/* ------------------------------------------------------------------ defaults (Sec. 4.1) */
void orc_default_params(orc_params* p) {
  memset(p, 0, sizeof(*p));
  p->tol = 1e-8;
  p->max_iter = 1000000;
  p->check_every = 100;
  p->restart_every = 10;
  p->alpha1 = 0.2;
  p->alpha2 = 0.8;
  p->alpha3 = 0.5;
  p->alpha3_tight = 0.2;
  p->ratio_tight = 0.1;
  p->lambda_A = 0.0;
  p->lambda_Q = 0.0;
  p->sigma0 = 0.0;
  p->power_max_iter = 5000;
  p->power_tol = 1e-6;
  p->power_safety = 1.01;
  p->scaling = 1;
}

static int bad_double(double v) { return isnan(v); }

/* [lo, hi] as the paper admits it (Sec. 1): lo in R u {-inf}, hi in R u {+inf}, lo <= hi */
static int bad_interval(double lo, double hi) {
  return bad_double(lo) || bad_double(hi) || lo > hi || lo == INFINITY || hi == -INFINITY;
}

static int validate(const orc_problem* P, const orc_params* prm) {
  if (P->n <= 0 || P->m < 0 || prm->max_iter < 1 || !(prm->tol > 0.0)) return 0;
  if (prm->check_every < 1 || prm->restart_every < 1) return 0;
  for (int64_t j = 0; j < P->n; j++) {
    if (!isfinite(P->c[j]) || bad_interval(P->L[j], P->U[j])) return 0;
  }
  for (int64_t i = 0; i < P->m; i++)
    if (bad_interval(P->l[i], P->u[i])) return 0;
  if (P->m > 0 && P->A_rowptr[0] != 0) return 0;
  for (int64_t i = 0; i < P->m; i++) {
    if (P->A_rowptr[i + 1] < P->A_rowptr[i]) return 0;
    for (int32_t k = P->A_rowptr[i]; k < P->A_rowptr[i + 1]; k++)
      if (P->A_colidx[k] < 0 || P->A_colidx[k] >= P->n || !isfinite(P->A_vals[k])) return 0;
  }
  if (P->phi != ORC_PHI_BOX && !(P->lambda >= 0.0)) return 0;
  return 1;
}


/* ------------------------------------------------------------------ preconditioning (Sec. 4.1)
 * The matrix that is equilibrated is K = [Q A^T; A 0] (symmetric, order n + m), scaled as
 * diag(s) K diag(s) with s = (d, e).  One pass computes the norm of every column of the
 * scaled K (the infinity norm in the 10 Ruiz passes, the 1-norm in the Pock-Chambolle pass
 * with alpha = 1) and divides s_j by the square root of it (columns of norm 0 keep s_j). */
static int scaling_eligible(const orc_problem* P) {
  if (P->phi != ORC_PHI_BOX) return 0;
  for (int32_t t = 0; t < P->nq; t++) {
    int32_t kd = P->q[t].kind;
    if (kd != ORC_Q_DIAG && kd != ORC_Q_CSR && kd != ORC_Q_DIA) return 0;
  }
  return 1;
}

/* accumulate |v| into the column norm (inf: max, one: sum) */
static void acc_norm(double* nrm, int64_t j, double v, int inf) {
  v = fabs(v);
  if (inf) nrm[j] = fmax(nrm[j], v);
  else nrm[j] += v;
}

static void scaled_col_norms(const orc_problem* P, const double* d, const double* e, int inf, double* cn,
                             double* rn) {
  int64_t n = P->n, m = P->m;
  for (int64_t j = 0; j < n; j++) cn[j] = 0.0;
  for (int64_t i = 0; i < m; i++) rn[i] = 0.0;
  for (int32_t t = 0; t < P->nq; t++) {
    const orc_qterm* T = &P->q[t];
    if (T->kind == ORC_Q_DIAG) {
      for (int64_t j = 0; j < n; j++) acc_norm(cn, j, T->dense[j] * d[j] * d[j], inf);
    } else if (T->kind == ORC_Q_CSR) {
      /* Q symmetric: the column norm of column j equals the norm of row j */
      for (int64_t i = 0; i < n; i++)
        for (int32_t k = T->rowptr[i]; k < T->rowptr[i + 1]; k++)
          acc_norm(cn, i, T->vals[k] * d[i] * d[T->colidx[k]], inf);
    } else { /* DIA: Q[i][i+o] and its mirror Q[i+o][i] */
      for (int32_t kk = 0; kk < T->ndiag; kk++) {
        int64_t o = T->offsets[kk];
        for (int64_t i = 0; i + o < n; i++) {
          double v = T->diags[(int64_t)kk * n + i] * d[i] * d[i + o];
          acc_norm(cn, i, v, inf);
          if (o != 0) acc_norm(cn, i + o, v, inf);
        }
      }
    }
  }
  /* A block (rows n..n+m of K) and its transpose (columns n..n+m) */
  for (int64_t i = 0; i < m; i++)
    for (int32_t k = P->A_rowptr[i]; k < P->A_rowptr[i + 1]; k++) {
      int64_t j = P->A_colidx[k];
      double v = P->A_vals[k] * e[i] * d[j];
      acc_norm(cn, j, v, inf);
      acc_norm(rn, i, v, inf);
    }
}

int orc_scaling(const orc_problem* P, double* d, double* e) {
  int64_t n = P->n, m = P->m;
  for (int64_t j = 0; j < n; j++) d[j] = 1.0;
  for (int64_t i = 0; i < m; i++) e[i] = 1.0;
  if (!scaling_eligible(P)) return 0;
  double *cn = vnew(n), *rn = vnew(m);
  for (int pass = 0; pass < 11; pass++) {
    int inf = pass < 10; /* 10 Ruiz passes, then Pock-Chambolle (alpha = 1) */
    scaled_col_norms(P, d, e, inf, cn, rn);
    for (int64_t j = 0; j < n; j++)
      if (cn[j] > 0.0) d[j] /= sqrt(cn[j]);
    for (int64_t i = 0; i < m; i++)
      if (rn[i] > 0.0) e[i] /= sqrt(rn[i]);
  }
  free(cn);
  free(rn);
  return 1;
}

/* ------------------------------------------------------------------ Algorithm 4 */
/* P: the problem the iteration runs on.  With preconditioning, P is the scaled problem and
 * P0, d, e the original and the scaling (x = D xs, y = E ys, z = D^{-1} zs): warm starts,
 * traces, the stopping test of Sec. 4.1 and the outputs are in the original space. */
static int solve_core(const orc_problem* P, const orc_params* prm, orc_result* res, double* xout,
                      double* yout, double* zout, double* wout, const orc_problem* P0, const double* d,
                      const double* e) {
  int64_t n = P->n, m = P->m;
  /* Sec. 4.1: lambda_A >= lambda_1(AA^*), lambda_Q >= lambda_1(Q) by the power method */
  double lamA = prm->lambda_A > 0.0 ? prm->lambda_A
                                    : orc_power_A(P, prm->power_max_iter, prm->power_tol, prm->power_safety);
  double lamQ = prm->lambda_Q > 0.0 ? prm->lambda_Q
                                    : orc_power_Q(P, prm->power_max_iter, prm->power_tol, prm->power_safety);
  if (m > 0 && !(lamA > 0.0)) lamA = 1.0; /* A = 0: any positive value is >= lambda_1 */
  /* Sec. 4.1: sigma0 = ||b||/||c|| when both lie in [1e-16, 1e16], else 1 */
  double sigma = prm->sigma0;
  if (!(sigma > 0.0)) {
    double bb = 0.0;
    for (int64_t i = 0; i < m; i++) {
      double bl = isfinite(P->l[i]) ? fabs(P->l[i]) : 0.0;
      double bu = isfinite(P->u[i]) ? fabs(P->u[i]) : 0.0;
      double b = fmax(bl, bu);
      bb += b * b;
    }
    double nb = sqrt(bb), nc = nrm2(P->c, n);
    sigma = (nb >= 1e-16 && nb <= 1e16 && nc >= 1e-16 && nc <= 1e16) ? nb / nc : 1.0;
  }
  res->lambda_A = lamA;
  res->lambda_Q = lamQ;

  double *x = vnew(n), *w = vnew(n), *y = vnew(m);
  double *x0 = vnew(n), *w0 = vnew(n), *y0 = vnew(m);
  double *xb = vnew(n), *wb = vnew(n), *yb = vnew(m), *zb = vnew(n), *wh = vnew(n);
  double *dx = vnew(n), *dw = vnew(n), *dy = vnew(m);
  /* Sec. 4.1: start at the origin; a warm start sets x, y and w = x (Q w* = Q x*) */
  if (prm->x0) {
    for (int64_t j = 0; j < n; j++) x[j] = w[j] = d ? prm->x0[j] / d[j] : prm->x0[j];
  }
  if (prm->y0 && m > 0)
    for (int64_t i = 0; i < m; i++) y[i] = e ? prm->y0[i] / e[i] : prm->y0[i];
  double *ux = vnew(n), *uy = vnew(m), *uz = vnew(n); /* original-space bar iterate */
  memcpy(x0, x, sizeof(double) * n);
  memcpy(w0, w, sizeof(double) * n);
  if (m > 0) memcpy(y0, y, sizeof(double) * m);

  int64_t k = 0, t = 0, r = 0;
  double R_r0 = 0.0, R_prev = 0.0, R_first = -1.0;
  double alpha3 = prm->alpha3;
  int status = ORC_MAX_ITER;
  double eta3[3] = {INFINITY, INFINITY, INFINITY}, pobj = NAN, dobj = NAN;

  for (;;) {
    orc_step(P, sigma, lamA, lamQ, y, w, x, yb, wb, zb, xb, wh);
    int64_t kd = k + 1;
    int rtest = (t == 0 || kd % prm->restart_every == 0);
    int ttest = (kd % prm->check_every == 0) || kd >= prm->max_iter;
    double R = NAN;
    if (rtest) {
      /* R~_{r,t} = ||u^{r,t} - ubar^{r,t+1}||_M (Sec. 3.2) */
      for (int64_t j = 0; j < n; j++) {
        dx[j] = x[j] - xb[j];
        dw[j] = w[j] - wb[j];
      }
      for (int64_t i = 0; i < m; i++) dy[i] = y[i] - yb[i];
      R = sqrt(fmax(0.0, orc_mnorm2(P, sigma, lamA, lamQ, dy, dw, dx)));
    }
    if (k < prm->trace_len) {
      if (prm->trace_x)
        for (int64_t j = 0; j < n; j++) prm->trace_x[k * n + j] = d ? d[j] * xb[j] : xb[j];
      if (prm->trace_w)
        for (int64_t j = 0; j < n; j++) prm->trace_w[k * n + j] = d ? d[j] * wb[j] : wb[j];
      if (prm->trace_y && m > 0)
        for (int64_t i = 0; i < m; i++) prm->trace_y[k * m + i] = e ? e[i] * yb[i] : yb[i];
      if (prm->trace_R) prm->trace_R[k] = R;
      if (prm->trace_sigma) prm->trace_sigma[k] = sigma;
      if (prm->trace_restart) prm->trace_restart[k] = 0;
    }
    if (ttest) {
      if (d) {
        for (int64_t j = 0; j < n; j++) {
          ux[j] = d[j] * xb[j];
          uz[j] = zb[j] / d[j];
        }
        for (int64_t i = 0; i < m; i++) uy[i] = e[i] * yb[i];
        orc_eta(P0, ux, uy, uz, eta3, &pobj, &dobj);
      } else {
        orc_eta(P, xb, yb, zb, eta3, &pobj, &dobj);
      }
      if (isnan(eta3[0]) || isnan(eta3[1]) || isnan(eta3[2]) || isinf(pobj) || isinf(dobj)) {
        status = ORC_NUMERICAL;
        k = kd;
        break;
      }
      /* tolerance ladder of Sec. 4: the first test at which 1e-4 and 1e-6 are met */
      if (res->iters_1e4 == 0 && fmax(eta3[0], fmax(eta3[1], eta3[2])) <= 1e-4) res->iters_1e4 = kd;
      if (res->iters_1e6 == 0 && fmax(eta3[0], fmax(eta3[1], eta3[2])) <= 1e-6) res->iters_1e6 = kd;
      if (fmax(eta3[0], fmax(eta3[1], eta3[2])) <= prm->tol) {
        status = ORC_CONVERGED;
        k = kd;
        break;
      }
      if (kd >= prm->max_iter) {
        status = ORC_MAX_ITER;
        k = kd;
        break;
      }
    }
    /* restart criteria (3.6)-(3.8), tested from the second inner step on */
    int restart = 0;
    if (rtest && !prm->restart_off) {
      if (t == 0) {
        R_r0 = R;
      } else {
        restart = (R <= prm->alpha1 * R_r0) || (R <= prm->alpha2 * R_r0 && R > R_prev) ||
                  ((double)(t + 1) >= alpha3 * (double)kd);
      }
      R_prev = R;
    }
    if (restart) {
      if (r == 0) R_first = R;
      double ratio = (R_first > 0.0) ? R / R_first : 0.0;
      if (!prm->sigma_fixed) {
        /* Algorithm 5 with theta~ of eq. (3.11) from ubar^{r,tau_r} - u^{r,0} */
        for (int64_t j = 0; j < n; j++) {
          dx[j] = xb[j] - x0[j];
          dw[j] = wb[j] - w0[j];
        }
        for (int64_t i = 0; i < m; i++) dy[i] = yb[i] - y0[i];
        double* Qdw = vnew(n);
        double* Atdy = vnew(n);
        double* QAtdy = vnew(n);
        orc_qmul(P, dw, Qdw);
        orc_atmul(P, dy, Atdy);
        orc_qmul(P, Atdy, QAtdy);
        double th1 = lamA * dot(dy, dy, m) + lamQ * dot(dw, Qdw, n) - 2.0 * dot(Qdw, Atdy, n);
        double th2 = dot(dx, dx, n);
        double th3 = dot(Atdy, QAtdy, n);
        free(Qdw);
        free(Atdy);
        free(QAtdy);
        sigma = orc_sigma_update(th1, th2, th3, lamQ, ratio, sigma, prm->sigma_golden);
      }
      if (ratio <= prm->ratio_tight) alpha3 = prm->alpha3_tight;
      /* u^{r+1,0} = ubar^{r,tau_r}: new anchor and new current point */
      memcpy(x, xb, sizeof(double) * n);
      memcpy(w, wb, sizeof(double) * n);
      memcpy(x0, xb, sizeof(double) * n);
      memcpy(w0, wb, sizeof(double) * n);
      if (m > 0) {
        memcpy(y, yb, sizeof(double) * m);
        memcpy(y0, yb, sizeof(double) * m);
      }
      t = 0;
      r++;
      if (k < prm->trace_len && prm->trace_restart) prm->trace_restart[k] = 1;
    } else {
      /* Halpern step: u = 1/(i+2) u^{r,0} + (i+1)/(i+2) (2 ubar - u), i = t (or k) */
      double i = prm->halpern_total ? (double)k : (double)t;
      double a = 1.0 / (i + 2.0), b = (i + 1.0) / (i + 2.0);
      for (int64_t j = 0; j < n; j++) {
        x[j] = a * x0[j] + b * (2.0 * xb[j] - x[j]);
        w[j] = a * w0[j] + b * (2.0 * wb[j] - w[j]);
      }
      for (int64_t i2 = 0; i2 < m; i2++) y[i2] = a * y0[i2] + b * (2.0 * yb[i2] - y[i2]);
      t++;
    }
    k = kd;
  }

  res->eta_p = eta3[0];
  res->eta_d = eta3[1];
  res->eta_gap = eta3[2];
  res->pobj = pobj;
  res->dobj = dobj;
  res->iters = k;
  res->restarts = r;
  res->sigma = sigma;
  res->status = status;
  for (int64_t j = 0; j < n; j++) {
    if (xout) xout[j] = d ? d[j] * xb[j] : xb[j];
    if (zout) zout[j] = d ? zb[j] / d[j] : zb[j];
    if (wout) wout[j] = d ? d[j] * wb[j] : wb[j];
  }
  if (yout)
    for (int64_t i = 0; i < m; i++) yout[i] = e ? e[i] * yb[i] : yb[i];
  free(ux); free(uy); free(uz);
  free(x); free(w); free(y); free(x0); free(w0); free(y0);
  free(xb); free(wb); free(yb); free(zb); free(wh);
  free(dx); free(dw); free(dy);
  return status;
}


/* ------------------------------------------------------------------ primal HPR (Appendix A)
 * Algorithm 6 (method 1) on min 1/2<x,Qx> + <c,x> + phi(x) + delta_K(s) s.t. Ax = s, with
 * S_x = lambda_Q I - Q + sigma (lambda_A I - A^*A), and Algorithm 7 (method 2) on the
 * reformulation with v = x, S_v = lambda_Q I - Q, S_x = sigma (lambda_A I - A^*A); both with
 * the Halpern step of Step 5, fixed sigma and no restarts, as printed.  The proximal terms
 * make the x-step separable:
 *   method 1:  tau = lambda_Q + sigma lambda_A,
 *              xbar = Prox_{phi/tau}(x - (Qx + c - A^*(2 ybar - y)) / tau)
 *   method 2:  vbar = (lambda_Q v - Qv + sigma x - t) / (lambda_Q + sigma),
 *              tau = sigma (1 + lambda_A),
 *              xbar = Prox_{phi/tau}(x - (c - A^*(2 ybar - y) - tbar + sigma (x - vbar)) / tau)
 * with sbar = Pi_K(Ax - y/sigma) and ybar = y + sigma (sbar - Ax) from Steps 1-2 (A^*(2 ybar - y)
 * = A^*(ybar + sigma (sbar - Ax))).  The multiplier of phi is zbar = tau (xbar - r) for the
 * prox argument r, so that the stopping rule of Sec. 4.1 is evaluated at (xbar, ybar, zbar). */
static int solve_primal(const orc_problem* P, const orc_params* prm, orc_result* res, double* xout, double* yout,
                        double* zout, double* wout) {
  int64_t n = P->n, m = P->m;
  const int two = prm->method == 2;
  double lamA = prm->lambda_A > 0.0 ? prm->lambda_A
                                    : orc_power_A(P, prm->power_max_iter, prm->power_tol, prm->power_safety);
  double lamQ = prm->lambda_Q > 0.0 ? prm->lambda_Q
                                    : orc_power_Q(P, prm->power_max_iter, prm->power_tol, prm->power_safety);
  if (m > 0 && !(lamA > 0.0)) lamA = 1.0;
  double sigma = prm->sigma0;
  if (!(sigma > 0.0)) {
    double bb = 0.0;
    for (int64_t i = 0; i < m; i++) {
      double bl = isfinite(P->l[i]) ? fabs(P->l[i]) : 0.0;
      double bu = isfinite(P->u[i]) ? fabs(P->u[i]) : 0.0;
      double b = fmax(bl, bu);
      bb += b * b;
    }
    double nb = sqrt(bb), nc = nrm2(P->c, n);
    sigma = (nb >= 1e-16 && nb <= 1e16 && nc >= 1e-16 && nc <= 1e16) ? nb / nc : 1.0;
  }
  res->lambda_A = lamA;
  res->lambda_Q = lamQ;
  const double tau = two ? sigma * (1.0 + lamA) : lamQ + sigma * lamA;
  double *x = vnew(n), *s = vnew(m), *y = vnew(m), *v = vnew(n), *t = vnew(n);
  double *x0 = vnew(n), *s0 = vnew(m), *y0 = vnew(m), *v0 = vnew(n), *t0 = vnew(n);
  double *xb = vnew(n), *sb = vnew(m), *yb = vnew(m), *vb = vnew(n), *tb = vnew(n), *zb = vnew(n);
  double *Ax = vnew(m), *Qv = vnew(n), *w = vnew(m), *ATw = vnew(n);
  if (prm->x0) {
    memcpy(x, prm->x0, sizeof(double) * n);
    memcpy(v, prm->x0, sizeof(double) * n);
  }
  if (prm->y0 && m > 0) memcpy(y, prm->y0, sizeof(double) * m);
  memcpy(x0, x, sizeof(double) * n);
  memcpy(v0, v, sizeof(double) * n);
  if (m > 0) memcpy(y0, y, sizeof(double) * m);
  int64_t k = 0;
  int status = ORC_MAX_ITER;
  double eta3[3] = {INFINITY, INFINITY, INFINITY}, pobj = NAN, dobj = NAN;
  for (;;) {
    orc_amul(P, x, Ax);
    orc_qmul(P, two ? v : x, Qv);
    for (int64_t i = 0; i < m; i++) {
      /* Steps 1-2: with q = Ax - y/sigma, sbar = Pi_K(q) and ybar = y + sigma (sbar - Ax)
       * = sigma (Pi_K(q) - q), evaluated in the second form so that ybar is exactly 0 on rows
       * where the projection is inactive (its sign then matches K exactly) */
      const double q = Ax[i] - y[i] / sigma;
      sb[i] = clampd(q, P->l[i], P->u[i]);
      yb[i] = sigma * (sb[i] - q);
      w[i] = 2.0 * yb[i] - y[i];
    }
    if (two)
      for (int64_t j = 0; j < n; j++) {
        vb[j] = (lamQ * v[j] - Qv[j] + sigma * x[j] - t[j]) / (lamQ + sigma);   /* Step 1 (v) */
        tb[j] = t[j] + sigma * (vb[j] - x[j]);                                  /* Step 2.2 */
      }
    orc_atmul(P, w, ATw);
    for (int64_t j = 0; j < n; j++) {                            /* Step 3 */
      double g = two ? P->c[j] - ATw[j] - tb[j] + sigma * (x[j] - vb[j]) : Qv[j] + P->c[j] - ATw[j];
      double r = x[j] - g / tau;
      xb[j] = prox_phi(P, j, r, 1.0 / tau);
      zb[j] = tau * (xb[j] - r);
    }
    int64_t kd = k + 1;
    if (k < prm->trace_len) {
      if (prm->trace_x) memcpy(prm->trace_x + k * n, xb, sizeof(double) * n);
      if (prm->trace_y && m > 0) memcpy(prm->trace_y + k * m, yb, sizeof(double) * m);
      if (prm->trace_sigma) prm->trace_sigma[k] = sigma;
    }
    if ((kd % prm->check_every == 0) || kd >= prm->max_iter) {
      orc_eta(P, xb, yb, zb, eta3, &pobj, &dobj);
      if (isnan(eta3[0]) || isnan(eta3[1]) || isnan(eta3[2]) || isinf(pobj) || isinf(dobj)) {
        status = ORC_NUMERICAL;
        k = kd;
        break;
      }
      if (res->iters_1e4 == 0 && fmax(eta3[0], fmax(eta3[1], eta3[2])) <= 1e-4) res->iters_1e4 = kd;
      if (res->iters_1e6 == 0 && fmax(eta3[0], fmax(eta3[1], eta3[2])) <= 1e-6) res->iters_1e6 = kd;
      if (fmax(eta3[0], fmax(eta3[1], eta3[2])) <= prm->tol) {
        status = ORC_CONVERGED;
        k = kd;
        break;
      }
      if (kd >= prm->max_iter) {
        k = kd;
        break;
      }
    }
    /* Steps 4-5: u = 1/(k+2) u^0 + (k+1)/(k+2) (2 ubar - u) */
    const double a = 1.0 / (k + 2.0), b = (k + 1.0) / (k + 2.0);
    for (int64_t j = 0; j < n; j++) {
      x[j] = a * x0[j] + b * (2.0 * xb[j] - x[j]);
      if (two) {
        v[j] = a * v0[j] + b * (2.0 * vb[j] - v[j]);
        t[j] = a * t0[j] + b * (2.0 * tb[j] - t[j]);
      }
    }
    for (int64_t i = 0; i < m; i++) {
      s[i] = a * s0[i] + b * (2.0 * sb[i] - s[i]);
      y[i] = a * y0[i] + b * (2.0 * yb[i] - y[i]);
    }
    k = kd;
  }
  res->eta_p = eta3[0];
  res->eta_d = eta3[1];
  res->eta_gap = eta3[2];
  res->pobj = pobj;
  res->dobj = dobj;
  res->iters = k;
  res->sigma = sigma;
  res->status = status;
  if (xout) memcpy(xout, xb, sizeof(double) * n);
  if (yout && m > 0) memcpy(yout, yb, sizeof(double) * m);
  if (zout) memcpy(zout, zb, sizeof(double) * n);
  if (wout) memcpy(wout, two ? vb : xb, sizeof(double) * n);
  free(x); free(s); free(y); free(v); free(t); free(x0); free(s0); free(y0); free(v0); free(t0);
  free(xb); free(sb); free(yb); free(vb); free(tb); free(zb); free(Ax); free(Qv); free(w); free(ATw);
  return status;
}

/* Algorithm 4, on the preconditioned problem when prm->scaling applies (Sec. 4.1): with
 * x = D xs and y = E ys the scaled data are A_s = E A D, Q_s = D Q D, c_s = D c,
 * [l_s, u_s] = E [l, u], [L_s, U_s] = D^{-1} [L, U]. */
int orc_solve(const orc_problem* P, const orc_params* prm, orc_result* res, double* xout,
              double* yout, double* zout, double* wout) {
  memset(res, 0, sizeof(*res));
  if (!validate(P, prm)) {
    res->status = ORC_INVALID;
    return ORC_INVALID;
  }
  if (prm->method == 1 || prm->method == 2) return solve_primal(P, prm, res, xout, yout, zout, wout);
  if (prm->method != 0) {
    res->status = ORC_INVALID;
    return ORC_INVALID;
  }
  if (!prm->scaling || !scaling_eligible(P)) return solve_core(P, prm, res, xout, yout, zout, wout, NULL, NULL, NULL);
  int64_t n = P->n, m = P->m;
  double *d = vnew(n), *e = vnew(m);
  orc_scaling(P, d, e);
  int64_t nnzA = m > 0 ? P->A_rowptr[m] : 0;
  double *Av = vnew(nnzA), *c = vnew(n), *L = vnew(n), *U = vnew(n), *l = vnew(m), *u = vnew(m);
  for (int64_t i = 0; i < m; i++)
    for (int32_t k = P->A_rowptr[i]; k < P->A_rowptr[i + 1]; k++) Av[k] = e[i] * P->A_vals[k] * d[P->A_colidx[k]];
  for (int64_t j = 0; j < n; j++) {
    c[j] = d[j] * P->c[j];
    L[j] = P->L[j] / d[j];
    U[j] = P->U[j] / d[j];
  }
  for (int64_t i = 0; i < m; i++) {
    l[i] = e[i] * P->l[i];
    u[i] = e[i] * P->u[i];
  }
  orc_qterm* q = (orc_qterm*)calloc((size_t)(P->nq > 0 ? P->nq : 1), sizeof(orc_qterm));
  double** qv = (double**)calloc((size_t)(P->nq > 0 ? P->nq : 1), sizeof(double*));
  for (int32_t t = 0; t < P->nq; t++) {
    const orc_qterm* T = &P->q[t];
    q[t] = *T;
    if (T->kind == ORC_Q_DIAG) {
      qv[t] = vnew(n);
      for (int64_t j = 0; j < n; j++) qv[t][j] = d[j] * T->dense[j] * d[j];
      q[t].dense = qv[t];
    } else if (T->kind == ORC_Q_CSR) {
      qv[t] = vnew(T->rowptr[n]);
      for (int64_t i = 0; i < n; i++)
        for (int32_t k = T->rowptr[i]; k < T->rowptr[i + 1]; k++) qv[t][k] = d[i] * T->vals[k] * d[T->colidx[k]];
      q[t].vals = qv[t];
    } else {
      qv[t] = vnew((int64_t)T->ndiag * n);
      for (int32_t kk = 0; kk < T->ndiag; kk++)
        for (int64_t i = 0; i + T->offsets[kk] < n; i++)
          qv[t][(int64_t)kk * n + i] = d[i] * T->diags[(int64_t)kk * n + i] * d[i + T->offsets[kk]];
      q[t].diags = qv[t];
    }
  }
  orc_problem S = *P;
  S.q = q;
  S.A_vals = Av;
  S.c = c;
  S.L = L;
  S.U = U;
  S.l = l;
  S.u = u;
  int st = solve_core(&S, prm, res, xout, yout, zout, wout, P, d, e);
  for (int32_t t = 0; t < P->nq; t++) free(qv[t]);
  free(qv); free(q);
  free(Av); free(c); free(L); free(U); free(l); free(u); free(d); free(e);
  return st;
}
