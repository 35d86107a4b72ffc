// Batched HPR-QP: many independent instances of eq. (1.1), one persistent launch per bucket of n.
//
// One thread block owns one instance at a time and runs Algorithm 4 on it to the end, with its
// own sigma, restart and termination state (Sec. 3.2-3.3, Sec. 4.1); blocks take instances from
// their bucket's atomic work queue, ordered by estimated cost, largest first.  No block ever
// waits on another.  The buckets' launches are queued on parallel streams, largest n first, so
// an SM whose block leaves an exhausted bucket starts blocks of the next one.  Per bucket the
// autotuner picks the block size (64 to 512 threads per instance) and whether a block keeps its
// instance's dense factor F in shared memory for the whole solve.
//
// Per inner step the only work of order k*n is Q xbar-type products through the dense factor
// (t = F v, then F^T t); everything else is elementwise or of order m*n with m <= 32:
//   * the second Q product of a step, Q wbar = Q wbar_{1/2} + s (Q A^T)(ybar - y), uses Q A^T
//     (n x m), formed once per solve (linearity of Q);
//   * theta_3 of R~ (eq. (2.12)) and theta~_3 of eq. (3.11) are quadratic forms with A Q A^T
//     (m x m), so a restart needs no pass over Q;
//   * A v is accumulated row by row over A's CSR rows in one block pass, A^T ybar from the
//     stored transpose (2 entries per row for the portfolio family).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/hprqp.h"
#include "kernels.cuh"

namespace hprqp {
namespace batch {

constexpr int kMaxM = HPRQP_BATCH_MAX_M;
constexpr int kMaxP = HPRQP_BATCH_MAX_P;

struct Inst {
  int64_t n, m, p;            // p: rows of the dense factor (0: none)
  int phi;
  double lambda;
  int64_t on;                 // offset into the n-pools
  int64_t om;                 // offset into the m-pools
  int64_t oF;                 // offset into the F pool
  int64_t oqat;               // offset into the (n*m) pool
  int64_t oaqa;               // offset into the (m*m) pool
  int64_t oarp, oann;         // A: row pointers (m+1), entries
  int64_t otrp, otnn;         // A^T: row pointers (n+1), entries
  int64_t oqrp, oqnn;         // Q CSR: row pointers (n+1), entries; oqrp < 0: none
  int has_diag;
  int has_ws;                 // warm start given
  double nb2, nc2, b_inf, c_inf;
  double lamA, lamQ, sigma0;  // > 0: given
};

struct Res {
  double eta_p, eta_d, eta_gap, pobj, dobj, sigma, lamA, lamQ;
  long long iters, restarts;
  int status;
  int pad;
};

// pools of the batch (device pointers)
struct Pools {
  const Inst* inst;
  Res* res;
  const int* order;
  unsigned* head;
  int count;
  // n-pools
  const double *c, *L, *U, *d, *x0in;
  double *x, *w, *Qw, *ATy, *x0, *w0, *Qw0, *ATy0, *xb, *wb, *Qwb, *ATyb, *wh, *Qwh, *v, *zb, *Qxb, *s1, *s2;
  // m-pools
  const double *l, *u, *y0in;
  double *y, *y0, *yb;
  const double* F;
  double *qat, *aqa;
  const int *arp, *aci, *trp, *tci, *qrp, *qci;
  const double *av, *tv, *qv;
  // algorithm parameters
  double tol, alpha1, alpha2, alpha3, alpha3_tight, ratio_tight, power_tol, power_safety;
  long long max_iter, check_every, restart_every, power_max_iter;
  int halpern_total, restart_off, sigma_fixed, sigma_golden;
};

// ------------------------------------------------------------------------------------ block helpers
template <int NT>
__device__ __forceinline__ void bsum(double (&v)[NT], unsigned maxmask, double* red) {
  block_reduce<NT>(v, maxmask, red);
  // thread 0 holds the result; broadcast through shared memory
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NT; i++) red[i] = v[i];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NT; i++) v[i] = red[i];
  __syncthreads();
}

// t[r] = sum_j F[r][j] x[j] (and F x1 when x1), one warp per row; result in shared t0/t1.  A
// warp streams one row at a time (consecutive addresses); wider forms that interleave several
// rows or unroll across rows measured slower on the large instances, whose F comes from HBM.
__device__ __forceinline__ void dense_fx(const double* __restrict__ F, int64_t p, int64_t n,
                                        const double* __restrict__ x0, const double* __restrict__ x1, double* t0,
                                        double* t1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t r = warp; r < p; r += nw) {
    const double* Fr = F + r * n;
    double s0 = 0.0, s1 = 0.0;
    for (int64_t j = lane; j < n; j += 32) {
      const double f = Fr[j];
      s0 = fma(f, x0[j], s0);
      if (x1) s1 = fma(f, x1[j], s1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, o);
      if (x1) s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      t0[r] = s0;
      if (x1) t1[r] = s1;
    }
  }
}

extern __shared__ __align__(16) unsigned char smem_raw[];
template <int PC>
struct Shared;

// The instance's dense factor F (p x n, row-major): in global memory, or (FS) the block's copy
// in shared memory after its Shared state.
template <bool FS, int PC>
__device__ __forceinline__ const double* fac(const Pools& P, const Inst& I) {
  if constexpr (FS) return reinterpret_cast<const double*>(smem_raw + sizeof(Shared<PC>));
  else return P.F + I.oF;
}

// (Q x)_j = sum_r F[r][j] t[r] + d_j x_j + (Q_csr x)_j for one coordinate
template <bool FS, int PC>
__device__ __forceinline__ double q_row(const Pools& P, const Inst& I, int64_t j, const double* __restrict__ x,
                                        const double* t) {
  double acc = 0.0;
  if (I.p) {
    const double* F = fac<FS, PC>(P, I);
    for (int64_t r = 0; r < I.p; r++) acc = fma(F[r * I.n + j], t[r], acc);
  }
  if (I.has_diag) acc = fma(P.d[I.on + j], x[j], acc);
  if (I.oqrp >= 0) {
    const int* rp = P.qrp + I.oqrp;
    const int* ci = P.qci + I.oqnn;
    const double* qv = P.qv + I.oqnn;
    for (int k = rp[j]; k < rp[j + 1]; k++) acc = fma(qv[k], x[ci[k]], acc);
  }
  return acc;
}

// out = Q x for the whole instance (x, out in global memory, x != out); t: shared scratch (p)
template <bool FS, int PC>
__device__ void block_qmul(const Pools& P, const Inst& I, const double* x, double* out, double* t) {
  if (I.p) dense_fx(fac<FS, PC>(P, I), I.p, I.n, x, nullptr, t, nullptr);
  __syncthreads();
  for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x) out[j] = q_row<FS, PC>(P, I, j, x, t);
  __syncthreads();
}

// (A v)_i for all rows i into shared av[m] (and A x1 into ax[m] when x1); block pass over the
// rows of A: per row, lanes stride its entries, warps combine in shared memory (fixed order)
__device__ void block_amul(const Pools& P, const Inst& I, const double* __restrict__ v, const double* __restrict__ x1,
                           double* av, double* ax, double* wred) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int* rp = P.arp + I.oarp;
  const int* ci = P.aci + I.oann;
  const double* a = P.av + I.oann;
  for (int64_t i = 0; i < I.m; i++) {
    double s0 = 0.0, s1 = 0.0;
    for (int k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x) {
      const double aik = a[k];
      s0 = fma(aik, v[ci[k]], s0);
      if (x1) s1 = fma(aik, x1[ci[k]], s1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_down_sync(0xffffffffu, s0, o);
      if (x1) s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      wred[i * 32 + warp] = s0;
      if (x1) wred[(kMaxM + i) * 32 + warp] = s1;
    }
  }
  __syncthreads();
  if (threadIdx.x < I.m) {
    double s0 = 0.0, s1 = 0.0;
    for (int q = 0; q < nw; q++) {
      s0 += wred[threadIdx.x * 32 + q];
      if (x1) s1 += wred[(kMaxM + threadIdx.x) * 32 + q];
    }
    av[threadIdx.x] = s0;
    if (x1) ax[threadIdx.x] = s1;
  }
  __syncthreads();
}

// (A^T y)_j with y in shared memory
__device__ __forceinline__ double at_row(const Pools& P, const Inst& I, int64_t j, const double* ys) {
  const int* rp = P.trp + I.otrp;
  const int* ci = P.tci + I.otnn;
  const double* tv = P.tv + I.otnn;
  double acc = 0.0;
  for (int k = rp[j]; k < rp[j + 1]; k++) acc = fma(tv[k], ys[ci[k]], acc);
  return acc;
}

// power method of Sec. 4.1 on Q (which = 1, R^n) or A A^* (which = 0, R^m); pv, pw, tmp: global
// scratch of the instance; returns safety * Rayleigh quotient (valid in every thread)
template <bool FS, int PC>
__device__ double block_power(const Pools& P, const Inst& I, int which, double* pv, double* pw, double* tmp,
                              double* t, double* av, double* wred, double* red) {
  const int64_t dim = which ? I.n : I.m;
  if (dim == 0) return 0.0;
  double s2[1] = {0.0};
  for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) {
    const uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
    const double val = 0.5 + (double)h / 4294967296.0;
    pw[i] = val;
    s2[0] = fma(val, val, s2[0]);
  }
  bsum<1>(s2, 0u, red);
  double scale = 1.0 / sqrt(s2[0]), lam = 0.0;
  __syncthreads();
  for (long long it = 0; it < P.power_max_iter; it++) {
    for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) pv[i] = pw[i] * scale;
    __syncthreads();
    double acc[2] = {0.0, 0.0};
    if (which) {
      block_qmul<FS, PC>(P, I, pv, pw, t);
      for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) {
        acc[0] = fma(pv[i], pw[i], acc[0]);
        acc[1] = fma(pw[i], pw[i], acc[1]);
      }
    } else {
      // w = A (A^T v): A^T v from the stored transpose, then the row pass of A
      for (int64_t j = threadIdx.x; j < I.n; j += blockDim.x) tmp[j] = at_row(P, I, j, pv);
      __syncthreads();
      block_amul(P, I, tmp, nullptr, av, nullptr, wred);
      for (int64_t i = threadIdx.x; i < dim; i += blockDim.x) {
        pw[i] = av[i];
        acc[0] = fma(pv[i], av[i], acc[0]);
        acc[1] = fma(av[i], av[i], acc[1]);
      }
    }
    bsum<2>(acc, 0u, red);
    const double nw = sqrt(acc[1]);
    if (nw == 0.0 || !isfinite(nw)) return 0.0;
    const bool conv = it > 0 && fabs(acc[0] - lam) <= P.power_tol * fabs(acc[0]);
    lam = acc[0];
    scale = 1.0 / nw;
    if (conv) break;
  }
  return P.power_safety * lam;
}

// ------------------------------------------------------------------------------------ the solve
constexpr int kTerms = 20;   // block-reduced terms of one step
// 0..4  R~: sum dx^2, dw.Qdw, Qdw.A*dy, (unused), dx.(A*dy - Qdw)
// 5..11 eta: max rd, max |A*ybar|, max |Qxbar|, xbar.Qxbar, c.xbar, |xbar|_1, phi*(-zbar)
// 12..15 theta~ (restart candidates): |xbar-x0|^2, (wbar-w0).(Qwbar-Qw0), (Qwbar-Qw0).(A*ybar-A*y0), (unused)
constexpr unsigned kMaxMask = (1u << 5) | (1u << 6) | (1u << 7);

// Block state in shared memory, at fixed offsets (the hot loops address it with constants):
// t = F v for up to PC factor rows (PC = 256 or HPRQP_BATCH_MAX_P), the m-vectors, the warp
// partials of a block of at most 16 warps, the controller.  With FS the block's copy of F
// follows it (dynamic shared memory).
template <int PC>
struct __align__(16) Shared {
  double t0[PC], t1[PC];
  double av[kMaxM], ax[kMaxM];
  double y[kMaxM], yb[kMaxM], y0[kMaxM], lo[kMaxM], hi[kMaxM];
  double wred[2 * kMaxM * 32];
  double red[kTerms * 32];
  double pm[2][kMaxM];   // power-method vectors on R^m
  Ctrl C;
  int inst;
};

template <bool FS, int PC>
__device__ void solve_one(const Pools& P, int idx, Shared<PC>& S) {
  const Inst I = P.inst[idx];
  const int64_t n = I.n, m = I.m;
  const int tid = threadIdx.x, nt = blockDim.x;
  // instance views
  const double *c = P.c + I.on, *L = P.L + I.on, *U = P.U + I.on;
  double *x = P.x + I.on, *w = P.w + I.on, *Qw = P.Qw + I.on, *ATy = P.ATy + I.on;
  double *x0 = P.x0 + I.on, *w0 = P.w0 + I.on, *Qw0 = P.Qw0 + I.on, *ATy0 = P.ATy0 + I.on;
  double *xb = P.xb + I.on, *wb = P.wb + I.on, *Qwb = P.Qwb + I.on, *ATyb = P.ATyb + I.on;
  double *wh = P.wh + I.on, *Qwh = P.Qwh + I.on, *v = P.v + I.on, *zb = P.zb + I.on, *Qxb = P.Qxb + I.on;
  double *s1 = P.s1 + I.on, *s2 = P.s2 + I.on;
  double* ybg = P.yb + I.om;
  double* qat = P.qat + I.oqat;   // [j*m + i] = (Q A^T)_{j i}
  double* aqa = P.aqa + I.oaqa;   // [i*m + l]
  Ctrl& C = S.C;
  if constexpr (FS) {
    // the block's copy of F, read by every product of the solve
    double* Fs = reinterpret_cast<double*>(smem_raw + sizeof(Shared<PC>));
    const double* Fg = P.F + I.oF;
    for (int64_t q = tid; q < I.p * n; q += nt) Fs[q] = Fg[q];
    __syncthreads();
  }

  // ---- set-up (counted in the solve, like the power method): Q A^T, A Q A^T, lambda, sigma0
  for (int64_t i = 0; i < m; i++) {
    // column i of A^T = row i of A, scattered into s1
    for (int64_t j = tid; j < n; j += nt) s1[j] = 0.0;
    __syncthreads();
    {
      const int* rp = P.arp + I.oarp;
      const int* ci = P.aci + I.oann;
      const double* a = P.av + I.oann;
      for (int k = rp[i] + tid; k < rp[i + 1]; k += nt) s1[ci[k]] = a[k];  // distinct columns per row
    }
    __syncthreads();
    block_qmul<FS, PC>(P, I, s1, s2, S.t0);
    for (int64_t j = tid; j < n; j += nt) qat[j * m + i] = s2[j];
    __syncthreads();
  }
  for (int64_t i = 0; i < m; i++) {
    // row i of A Q A^T: A applied to column i of Q A^T
    for (int64_t j = tid; j < n; j += nt) s1[j] = qat[j * m + i];
    __syncthreads();
    block_amul(P, I, s1, nullptr, S.av, nullptr, S.wred);
    if (tid < m) aqa[tid * m + i] = S.av[tid];
    __syncthreads();
  }
  double lamA = I.lamA, lamQ = I.lamQ;
  if (m > 0 && !(lamA > 0.0)) lamA = block_power<FS, PC>(P, I, 0, S.pm[0], S.pm[1], v, S.t0, S.av, S.wred, S.red);
  if (m > 0 && !(lamA > 0.0)) lamA = 1.0;
  if (m == 0) lamA = 0.0;
  const bool HQ = I.p || I.has_diag || I.oqrp >= 0;
  if (HQ && !(lamQ > 0.0)) lamQ = block_power<FS, PC>(P, I, 1, s1, s2, v, S.t0, S.av, S.wred, S.red);
  if (!HQ) lamQ = 0.0;
  double sigma = I.sigma0;
  if (!(sigma > 0.0)) {
    const double nb = sqrt(I.nb2), nc = sqrt(I.nc2);
    sigma = (nb >= 1e-16 && nb <= 1e16 && nc >= 1e-16 && nc <= 1e16) ? nb / nc : 1.0;
  }
  // ---- starting point: origin or warm start (w = x), images Q w, A^* y
  for (int64_t j = tid; j < n; j += nt) {
    const double xv = I.has_ws ? P.x0in[I.on + j] : 0.0;
    x[j] = xv;
    w[j] = xv;
    x0[j] = xv;
    w0[j] = xv;
  }
  if (tid < m) {
    const double yv = I.has_ws ? P.y0in[I.om + tid] : 0.0;
    S.y[tid] = yv;
    S.y0[tid] = yv;
    S.yb[tid] = 0.0;
    S.lo[tid] = P.l[I.om + tid];
    S.hi[tid] = P.u[I.om + tid];
  }
  __syncthreads();
  if (I.has_ws) {
    block_qmul<FS, PC>(P, I, x, Qw, S.t0);
  } else {
    for (int64_t j = tid; j < n; j += nt) Qw[j] = 0.0;
  }
  for (int64_t j = tid; j < n; j += nt) {
    Qw0[j] = Qw[j];
    const double a = m > 0 ? at_row(P, I, j, S.y) : 0.0;
    ATy[j] = a;
    ATy0[j] = a;
  }
  if (tid == 0) {
    memset(&C, 0, sizeof(Ctrl));
    C.lamA = lamA;
    C.lamQ = lamQ;
    C.lambda = I.lambda;
    C.tol = P.tol;
    C.alpha1 = P.alpha1;
    C.alpha2 = P.alpha2;
    C.alpha3 = P.alpha3;
    C.alpha3_tight = P.alpha3_tight;
    C.ratio_tight = P.ratio_tight;
    C.c_inf = I.c_inf;
    C.b_inf = I.b_inf;
    C.max_iter = P.max_iter;
    C.check_every = P.check_every;
    C.restart_every = P.restart_every;
    C.halpern_total = P.halpern_total;
    C.restart_off = P.restart_off;
    C.sigma_fixed = P.sigma_fixed;
    C.sigma_golden = P.sigma_golden;
    C.has_A = m > 0;
    C.has_Q = HQ;
    C.phi = I.phi;
    C.R_first = -1.0;
    C.rtest = !C.restart_off;
    C.ttest = (1 % C.check_every == 0) || (1 >= C.max_iter);
    C.status = 1;
    set_sigma(C, sigma);
  }
  __syncthreads();

  // ---- Algorithm 4
  while (!C.done) {
    const int mode = C.mode;
    const double ha = C.ha, hb = C.hb, sg = C.sigma, c1 = C.c1, c2 = C.c2, tau = C.tau, isg = C.inv_sigma;
    const double sq = C.s, slA = C.slA, islA = C.inv_slA;
    const bool rtest = C.rtest, ttest = C.ttest;
    // P1: Halpern/restart update, eqs. (3.1)-(3.3)
    for (int64_t j = tid; j < n; j += nt) {
      double xv, wv = 0.0, qw = 0.0, aty = 0.0;
      if (mode == 1) {
        xv = fma(hb, fma(2.0, xb[j], -x[j]), ha * x0[j]);
        x[j] = xv;
        if (HQ) {
          wv = fma(hb, fma(2.0, wb[j], -w[j]), ha * w0[j]);
          qw = fma(hb, fma(2.0, Qwb[j], -Qw[j]), ha * Qw0[j]);
          w[j] = wv;
          Qw[j] = qw;
        }
        if (m > 0) {
          aty = fma(hb, fma(2.0, ATyb[j], -ATy[j]), ha * ATy0[j]);
          ATy[j] = aty;
        }
      } else if (mode == 2) {
        xv = xb[j];
        x[j] = xv;
        x0[j] = xv;
        if (HQ) {
          wv = wb[j];
          qw = Qwb[j];
          w[j] = wv;
          w0[j] = wv;
          Qw[j] = qw;
          Qw0[j] = qw;
        }
        if (m > 0) {
          aty = ATyb[j];
          ATy[j] = aty;
          ATy0[j] = aty;
        }
      } else {
        xv = x[j];
        wv = w[j];
        qw = Qw[j];
        aty = ATy[j];
      }
      double g = -c[j];
      if (HQ) g -= qw;
      if (m > 0) g += aty;
      const double rz = fma(sg, g, xv);
      const double xbar = prox_phi(I.phi, rz, L[j], U[j], tau);
      xb[j] = xbar;
      if (ttest) zb[j] = (xbar - rz) * isg;
      const double xh = fma(2.0, xbar, -xv);
      wh[j] = HQ ? fma(c2, xh, c1 * wv) : 0.0;
      v[j] = xh;   // Q = 0: v = what
    }
    if (tid < m) {
      // Halpern / restart on y (m <= 32: one thread per row)
      double yv = S.y[tid];
      if (mode == 1) yv = fma(hb, fma(2.0, S.yb[tid], -yv), ha * S.y0[tid]);
      else if (mode == 2) {
        yv = S.yb[tid];
        S.y0[tid] = yv;
      }
      S.y[tid] = yv;
    }
    __syncthreads();
    // P2-P3: Q wbar_{1/2} (+ Q xbar), v = what + sigma (Q w - Q wbar_{1/2})
    if (HQ) {
      if (I.p) dense_fx(fac<FS, PC>(P, I), I.p, n, wh, ttest ? xb : nullptr, S.t0, S.t1);
      __syncthreads();
      for (int64_t j = tid; j < n; j += nt) {
        const double qwh = q_row<FS, PC>(P, I, j, wh, S.t0);
        Qwh[j] = qwh;
        if (ttest) Qxb[j] = q_row<FS, PC>(P, I, j, xb, S.t1);
        if (m > 0) v[j] = fma(sg, Qw[j] - qwh, v[j]);
      }
      __syncthreads();
    }
    double T[kTerms];
#pragma unroll
    for (int q = 0; q < kTerms; q++) T[q] = 0.0;
    // P4: A v (+ A xbar), eq. (3.5) on the m rows
    if (m > 0) {
      block_amul(P, I, v, ttest ? xb : nullptr, S.av, S.ax, S.wred);
      if (tid < m) {
        const double yv = S.y[tid], lo = S.lo[tid], hi = S.hi[tid];
        const double ry = fma(-slA, yv, S.av[tid]);
        const double ybv = (iclamp(ry, lo, hi) - ry) * islA;
        S.yb[tid] = ybv;
        ybg[tid] = ybv;
      }
      __syncthreads();
    }
    // P5: A^* ybar, wbar (eq. (3.3)), Q wbar by linearity, the R~ / eta / theta~ sums
    for (int64_t j = tid; j < n; j += nt) {
      double atyb = 0.0, dq = 0.0;
      if (m > 0) {
        atyb = at_row(P, I, j, S.yb);
        ATyb[j] = atyb;
        if (HQ) {
          const double* qa = qat + j * m;
          for (int64_t i = 0; i < m; i++) dq = fma(qa[i], S.yb[i] - S.y[i], dq);
        }
      }
      double wbv = 0.0, qwb = 0.0;
      if (HQ) {
        wbv = m > 0 ? fma(sq, atyb - ATy[j], wh[j]) : wh[j];
        qwb = m > 0 ? fma(sq, dq, Qwh[j]) : Qwh[j];
        wb[j] = wbv;
        Qwb[j] = qwb;
      }
      if (rtest) {
        const double xbj = xb[j];
        const double dx = x[j] - xbj;
        const double qdw = HQ ? Qw[j] - qwb : 0.0;
        const double ady = m > 0 ? ATy[j] - atyb : 0.0;
        T[0] = fma(dx, dx, T[0]);
        if (HQ) T[1] = fma(w[j] - wbv, qdw, T[1]);
        T[2] = fma(qdw, ady, T[2]);
        T[4] = fma(dx, ady - qdw, T[4]);
        // theta~ candidates from ubar - u^{r,0} (used only if this step restarts)
        const double ex = xbj - x0[j];
        T[12] = fma(ex, ex, T[12]);
        if (HQ) {
          const double qe = qwb - Qw0[j];
          T[13] = fma(wbv - w0[j], qe, T[13]);
          T[14] = fma(qe, atyb - ATy0[j], T[14]);
        }
      }
      if (ttest) {
        const double xbj = xb[j], qxb = HQ ? Qxb[j] : 0.0, cj = c[j];
        T[5] = imax(T[5], iabs(atyb - qxb + zb[j] - cj));
        T[6] = imax(T[6], iabs(atyb));
        T[7] = imax(T[7], iabs(qxb));
        T[8] = fma(xbj, qxb, T[8]);
        T[9] = fma(cj, xbj, T[9]);
        if (I.phi != PHI_BOX) T[10] += iabs(xbj);
        T[11] += conj_phi_term(I.phi, zb[j], L[j], U[j], I.lambda);
      }
    }
    if (rtest || ttest) block_reduce<kTerms>(T, kMaxMask, S.red);
    __syncthreads();
    // P6: controller (one thread)
    if (tid == 0) {
      double Ls[kWL], P3[kW3];
#pragma unroll
      for (int q = 0; q < kWL; q++) Ls[q] = T[q];
      P3[0] = P3[1] = P3[2] = P3[3] = 0.0;
      double th3 = 0.0, th3r = 0.0, dyr2 = 0.0;
      for (int64_t i = 0; i < m; i++) {
        const double dy = S.y[i] - S.yb[i];
        const double dr = S.yb[i] - S.y0[i];
        P3[0] = fma(dy, dy, P3[0]);
        dyr2 = fma(dr, dr, dyr2);
        if (ttest) {
          const double ax = S.ax[i], lo = S.lo[i], hi = S.hi[i], ybv = S.yb[i];
          P3[1] = fmax(P3[1], fabs(ax - fmin(fmax(ax, lo), hi)));
          P3[2] = fmax(P3[2], fabs(ax));
          if (ybv > 0.0) P3[3] += lo * ybv;
          else if (ybv < 0.0) P3[3] += hi * ybv;
        }
        if (HQ) {
          double qd = 0.0, qr = 0.0;
          for (int64_t l2 = 0; l2 < m; l2++) {
            qd = fma(aqa[i * m + l2], S.y[l2] - S.yb[l2], qd);
            qr = fma(aqa[i * m + l2], S.yb[l2] - S.y0[l2], qr);
          }
          th3 = fma(dy, qd, th3);
          th3r = fma(dr, qr, th3r);
        }
      }
      // the single-instance controller expects s * theta_3 in Ls[3]
      Ls[3] = C.s * th3;
      const long long r_before = C.r;
      controller(C, Ls, P3);
      if (C.restart_pending) {
        // Algorithm 5 with theta~ of eq. (3.11) from ubar^{r,tau_r} - u^{r,0}
        double t1 = C.lamA * dyr2 + C.lamQ * T[13] - 2.0 * T[14];
        double t2 = T[12];
        t1 = fmax(t1, 1e-12);
        t2 = fmax(t2, 1e-12);
        double snew;
        sigma_argmin_dev(t1, t2, th3r, C.lamQ, C.sigma_golden, &snew);
        const double beta = exp(-C.ratio);
        const double sgn = exp(beta * log(snew) + (1.0 - beta) * log(C.sigma));
        if (!isfinite(sgn) || !(sgn > 0.0)) {
          C.status = 3;
          C.done = 1;
        } else {
          set_sigma(C, sgn);
        }
        C.restart_pending = 0;
      }
      (void)r_before;
    }
    __syncthreads();
  }
  // ---- results
  if (tid == 0) {
    Res R;
    R.eta_p = C.eta_p;
    R.eta_d = C.eta_d;
    R.eta_gap = C.eta_gap;
    R.pobj = C.pobj;
    R.dobj = C.dobj;
    R.sigma = C.sigma;
    R.lamA = C.lamA;
    R.lamQ = C.lamQ;
    R.iters = C.k;
    R.restarts = C.r;
    R.status = C.status;
    R.pad = 0;
    P.res[idx] = R;
  }
  __syncthreads();
}

// One bucket of instances: order[beg .. beg + count), taken from the work counter *head.
struct Bucket {
  int beg, count;
  unsigned* head;
};

// One block per instance at a time, blocks of any size from 64 to 512 threads (the autotuner's
// choice for the bucket); a block that finds the bucket's counter exhausted exits, and its SM
// takes blocks of the next bucket's launch (launched behind this one on another stream).
// Registers are capped at 64 so that 32 warps fit an SM (two 512-thread blocks): the dense-factor
// passes wait on memory, and twice the warps in flight outweigh the few spilled values (on the
// 4096-instance batch: 13.7 s against 14.9 s at 128 registers and 16 warps).
template <bool FS, int PC>
__global__ void __launch_bounds__(512, 2) k_batch(Pools P, Bucket B) {
  Shared<PC>& S = *reinterpret_cast<Shared<PC>*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned q = atomicAdd(B.head, 1u);
      S.inst = q < (unsigned)B.count ? P.order[B.beg + q] : -1;
    }
    __syncthreads();
    const int idx = S.inst;
    if (idx < 0) break;
    solve_one<FS, PC>(P, idx, S);
  }
}

// The four instantiations: the capacity of t (factor rows) and the shared-memory F copy.
constexpr int kSmallP = 256;
using KFn = void (*)(Pools, Bucket);
inline KFn batch_kernel(bool fs, bool small_p) {
  return small_p ? (fs ? k_batch<true, kSmallP> : k_batch<false, kSmallP>)
                 : (fs ? k_batch<true, kMaxP> : k_batch<false, kMaxP>);
}
inline size_t shared_bytes(bool small_p) { return small_p ? sizeof(Shared<kSmallP>) : sizeof(Shared<kMaxP>); }

}  // namespace batch
}  // namespace hprqp

// ======================================================================================= host side
using namespace hprqp;
using namespace hprqp::batch;

// Instances are bucketed by n, largest first; each bucket runs as its own launch, with the block
// size and the shared-memory F copy the autotuner chose for it.
constexpr int kMaxBuckets = 4;
struct Sched {
  int beg[kMaxBuckets + 1];    // bucket k: order[beg[k] .. beg[k+1])
  int64_t pmax[kMaxBuckets];   // largest p of the bucket
  int64_t fmax[kMaxBuckets];   // largest p*n of the bucket
  int threads[kMaxBuckets];    // block size (threads per instance)
  bool fs[kMaxBuckets];        // F copied to shared memory
};

struct hprqp_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hprqp_params prm;
  int count = 0;
  std::vector<Inst> hinst;
  std::vector<int64_t> n_of, m_of;
  Pools P;
  std::vector<void*> allocs;
  // schedule: instances bucketed by n (order sorted by bucket, then cost); per bucket the block
  // size and the shared-memory F copy, chosen by the autotuner at the first solve
  Sched sched;
  cudaStream_t side[kMaxBuckets - 1] = {};    // buckets 1.. run on these, behind bucket 0
  cudaEvent_t fork = nullptr, join[kMaxBuckets - 1] = {};
  std::vector<int> bucket_lo;   // smallest n of each bucket
  std::vector<int> horder;      // host copy of the work order
  bool tuned = false;
  std::vector<Res> hres;
  std::string err;
  double seconds = 0.0;
  int64_t launches = 0;
  bool solved = false;
};

static thread_local std::string g_batch_err;

static hprqp_status bfail(hprqp_batch* b, hprqp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  else g_batch_err = buf;
  return st;
}

#define BCU(b, call)                                                                                     \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) {                                                                             \
      cudaGetLastError();                                                                                \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? HPRQP_OOM : HPRQP_CUDA_ERROR, "%s: %s", #call, \
                   cudaGetErrorString(e_));                                                              \
    }                                                                                                    \
  } while (0)

static bool bdev(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
static hprqp_status bfetch(hprqp_batch* b, std::vector<T>& dst, const T* p, size_t cnt) {
  size_t old = dst.size();
  dst.resize(old + cnt);
  if (cnt == 0) return HPRQP_OK;
  if (!p) return bfail(b, HPRQP_INVALID_ARG, "null input pointer");
  if (bdev(p)) BCU(b, cudaMemcpy(dst.data() + old, p, cnt * sizeof(T), cudaMemcpyDeviceToHost));
  else std::memcpy(dst.data() + old, p, cnt * sizeof(T));
  return HPRQP_OK;
}

template <class T>
static hprqp_status bupload(hprqp_batch* b, T** out, const std::vector<T>& v) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  if (b->prm.alloc) {
    p = b->prm.alloc(bytes, b->prm.alloc_ctx, b->stream);
    if (!p) return bfail(b, HPRQP_OOM, "allocator hook failed");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, HPRQP_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  b->allocs.push_back(p);
  if (!v.empty()) BCU(b, cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, b->stream));
  else BCU(b, cudaMemsetAsync(p, 0, bytes, b->stream));
  *out = (T*)p;
  return HPRQP_OK;
}

static hprqp_status bzeros(hprqp_batch* b, double** out, size_t cnt) {
  void* p = nullptr;
  size_t bytes = std::max<size_t>(cnt, 1) * sizeof(double);
  if (b->prm.alloc) {
    p = b->prm.alloc(bytes, b->prm.alloc_ctx, b->stream);
    if (!p) return bfail(b, HPRQP_OOM, "allocator hook failed");
  } else {
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, HPRQP_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  b->allocs.push_back(p);
  BCU(b, cudaMemsetAsync(p, 0, bytes, b->stream));
  *out = (double*)p;
  return HPRQP_OK;
}

static void brelease(hprqp_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < kMaxBuckets - 1; k++) {
    if (b->side[k]) {
      cudaStreamSynchronize(b->side[k]);
      cudaStreamDestroy(b->side[k]);
    }
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  for (void* p : b->allocs) {
    if (b->prm.free) b->prm.free(p, 0, b->prm.alloc_ctx, b->stream);
    else cudaFree(p);
  }
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaGetLastError();
  delete b;
}

static hprqp_status batch_create_impl(hprqp_batch* b, int32_t count, const hprqp_problem* probs) {
  hprqp_status st;
  b->count = count;
  std::vector<double> c, L, U, d, x0in, l, u, y0in, F;
  std::vector<int> arp, aci, trp, tci, qrp, qci;
  std::vector<double> av, tv, qv;
  int64_t qat_total = 0, aqa_total = 0;
  b->hinst.resize(count);
  for (int32_t i = 0; i < count; i++) {
    const hprqp_problem& pr = probs[i];
    Inst I;
    std::memset(&I, 0, sizeof(I));
    const int64_t n = pr.n, m = pr.m;
    if (n <= 0 || m < 0 || m > kMaxM || n >= (int64_t)1 << 31)
      return bfail(b, HPRQP_INVALID_ARG, "instance %d: need n > 0 and 0 <= m <= %d", i, kMaxM);
    if (pr.phi < 0 || pr.phi > 2) return bfail(b, HPRQP_INVALID_ARG, "instance %d: bad phi", i);
    I.n = n;
    I.m = m;
    I.phi = pr.phi;
    I.lambda = pr.phi == 0 ? 0.0 : pr.lambda;
    if (pr.phi != 0 && !(pr.lambda >= 0.0 && std::isfinite(pr.lambda)))
      return bfail(b, HPRQP_INVALID_ARG, "instance %d: bad lambda", i);
    I.on = (int64_t)c.size();
    I.om = (int64_t)l.size();
    if ((st = bfetch(b, c, pr.c, n))) return st;
    if (pr.L && pr.phi != 1) {
      if ((st = bfetch(b, L, pr.L, n))) return st;
    } else {
      if (pr.phi != 1) return bfail(b, HPRQP_INVALID_ARG, "instance %d: L required", i);
      L.insert(L.end(), n, -INFINITY);
    }
    if (pr.U && pr.phi != 1) {
      if ((st = bfetch(b, U, pr.U, n))) return st;
    } else {
      if (pr.phi != 1) return bfail(b, HPRQP_INVALID_ARG, "instance %d: U required", i);
      U.insert(U.end(), n, INFINITY);
    }
    if ((st = bfetch(b, l, pr.l, m))) return st;
    if ((st = bfetch(b, u, pr.u, m))) return st;
    double nc2 = 0, ci = 0, nb2 = 0, bi = 0;
    for (int64_t j = 0; j < n; j++) {
      const double cj = c[I.on + j], Lj = L[I.on + j], Uj = U[I.on + j];
      if (!std::isfinite(cj) || std::isnan(Lj) || std::isnan(Uj) || Lj > Uj || Lj == INFINITY || Uj == -INFINITY)
        return bfail(b, HPRQP_INVALID_ARG, "instance %d: bad c or box at %lld", i, (long long)j);
      nc2 += cj * cj;
      ci = std::max(ci, std::fabs(cj));
    }
    for (int64_t r = 0; r < m; r++) {
      const double lr = l[I.om + r], ur = u[I.om + r];
      if (std::isnan(lr) || std::isnan(ur) || lr > ur || lr == INFINITY || ur == -INFINITY)
        return bfail(b, HPRQP_INVALID_ARG, "instance %d: bad row bounds", i);
      const double bb = std::max(std::isfinite(lr) ? std::fabs(lr) : 0.0, std::isfinite(ur) ? std::fabs(ur) : 0.0);
      nb2 += bb * bb;
      bi = std::max(bi, bb);
    }
    I.nb2 = nb2;
    I.nc2 = nc2;
    I.b_inf = bi;
    I.c_inf = ci;
    // warm start
    if (pr.x0) {
      I.has_ws = 1;
      if ((st = bfetch(b, x0in, pr.x0, n))) return st;
      if (m) {
        if (pr.y0) {
          if ((st = bfetch(b, y0in, pr.y0, m))) return st;
        } else {
          y0in.insert(y0in.end(), m, 0.0);
        }
      }
    } else {
      x0in.insert(x0in.end(), n, 0.0);
      y0in.insert(y0in.end(), m, 0.0);
    }
    I.sigma0 = pr.sigma0 > 0 && std::isfinite(pr.sigma0) ? pr.sigma0 : 0.0;
    I.lamA = pr.lambda_A > 0 ? pr.lambda_A : 0.0;
    I.lamQ = pr.lambda_Q > 0 ? pr.lambda_Q : 0.0;
    // A and its transpose
    std::vector<int> rp, cidx;
    std::vector<double> vals;
    if (m > 0) {
      if ((st = bfetch(b, rp, pr.A_rowptr, m + 1))) return st;
      if (rp[0] != 0) return bfail(b, HPRQP_INVALID_ARG, "instance %d: A row pointers", i);
      for (int64_t r = 0; r < m; r++)
        if (rp[r + 1] < rp[r]) return bfail(b, HPRQP_INVALID_ARG, "instance %d: A row pointers", i);
      if ((st = bfetch(b, cidx, pr.A_colidx, rp[m]))) return st;
      if ((st = bfetch(b, vals, pr.A_vals, rp[m]))) return st;
      for (int k = 0; k < rp[m]; k++)
        if (cidx[k] < 0 || cidx[k] >= n || !std::isfinite(vals[k]))
          return bfail(b, HPRQP_INVALID_ARG, "instance %d: A entries", i);
      // distinct columns inside each row (the Q A^T set-up scatters one row at a time)
      std::vector<int64_t> seen(n, -1);
      for (int64_t r = 0; r < m; r++)
        for (int k = rp[r]; k < rp[r + 1]; k++) {
          if (seen[cidx[k]] == r) return bfail(b, HPRQP_INVALID_ARG, "instance %d: duplicate entry in A row", i);
          seen[cidx[k]] = r;
        }
    } else {
      rp.assign(1, 0);
    }
    I.oarp = (int64_t)arp.size();
    I.oann = (int64_t)aci.size();
    arp.insert(arp.end(), rp.begin(), rp.end());
    aci.insert(aci.end(), cidx.begin(), cidx.end());
    av.insert(av.end(), vals.begin(), vals.end());
    {
      std::vector<int> trow(n + 1, 0);
      for (int k = 0; k < rp[m]; k++) trow[cidx[k] + 1]++;
      for (int64_t j = 0; j < n; j++) trow[j + 1] += trow[j];
      std::vector<int> pos(trow.begin(), trow.end() - 1), tcol(rp[m]);
      std::vector<double> tval(rp[m]);
      for (int64_t r = 0; r < m; r++)
        for (int k = rp[r]; k < rp[r + 1]; k++) {
          tcol[pos[cidx[k]]] = (int)r;
          tval[pos[cidx[k]]++] = vals[k];
        }
      I.otrp = (int64_t)trp.size();
      I.otnn = (int64_t)tci.size();
      trp.insert(trp.end(), trow.begin(), trow.end());
      tci.insert(tci.end(), tcol.begin(), tcol.end());
      tv.insert(tv.end(), tval.begin(), tval.end());
    }
    // Q
    I.oqrp = -1;
    const int nterms = pr.Q ? pr.Q->nterms : 0;
    bool seen_diag = false, seen_dense = false, seen_csr = false;
    for (int t = 0; t < nterms; t++) {
      const hprqp_qterm& q = pr.Q->terms[t];
      if (q.kind == HPRQP_Q_DIAG && !seen_diag) {
        seen_diag = true;
        I.has_diag = 1;
        if ((st = bfetch(b, d, q.dense, n))) return st;
        for (int64_t j = 0; j < n; j++)
          if (!std::isfinite(d[I.on + j])) return bfail(b, HPRQP_INVALID_ARG, "instance %d: Q diag", i);
      } else if (q.kind == HPRQP_Q_DENSE_FACTOR && !seen_dense) {
        seen_dense = true;
        if (q.p <= 0 || q.p > kMaxP) return bfail(b, HPRQP_INVALID_ARG, "instance %d: dense factor rows must be 1..%d", i, kMaxP);
        I.p = q.p;
        I.oF = (int64_t)F.size();
        if ((st = bfetch(b, F, q.dense, (size_t)q.p * n))) return st;
        for (size_t k = I.oF; k < F.size(); k++)
          if (!std::isfinite(F[k])) return bfail(b, HPRQP_INVALID_ARG, "instance %d: Q dense factor", i);
      } else if (q.kind == HPRQP_Q_CSR && !seen_csr) {
        seen_csr = true;
        std::vector<int> qr, qc;
        std::vector<double> qvv;
        if ((st = bfetch(b, qr, q.rowptr, n + 1))) return st;
        if (qr[0] != 0) return bfail(b, HPRQP_INVALID_ARG, "instance %d: Q csr", i);
        for (int64_t j = 0; j < n; j++)
          if (qr[j + 1] < qr[j]) return bfail(b, HPRQP_INVALID_ARG, "instance %d: Q csr", i);
        if ((st = bfetch(b, qc, q.colidx, qr[n]))) return st;
        if ((st = bfetch(b, qvv, q.vals, qr[n]))) return st;
        for (int k = 0; k < qr[n]; k++)
          if (qc[k] < 0 || qc[k] >= n || !std::isfinite(qvv[k])) return bfail(b, HPRQP_INVALID_ARG, "instance %d: Q csr", i);
        I.oqrp = (int64_t)qrp.size();
        I.oqnn = (int64_t)qci.size();
        qrp.insert(qrp.end(), qr.begin(), qr.end());
        qci.insert(qci.end(), qc.begin(), qc.end());
        qv.insert(qv.end(), qvv.begin(), qvv.end());
      } else {
        return bfail(b, HPRQP_INVALID_ARG, "instance %d: unsupported Q term (batched: one DIAG, one DENSE_FACTOR, one CSR)", i);
      }
    }
    if (!seen_diag) d.insert(d.end(), n, 0.0);
    I.oqat = qat_total;
    qat_total += n * m;
    I.oaqa = aqa_total;
    aqa_total += m * m;
    b->hinst[i] = I;
    b->n_of.push_back(n);
    b->m_of.push_back(m);
  }
  // buckets by n (largest first), and inside a bucket the largest estimated cost first (dense
  // factor passes, else n): every block takes the next instance of its bucket from a counter
  static const int64_t kBucketLo[kMaxBuckets] = {3000, 1500, 600, 0};
  auto bucket_of = [](int64_t n) {
    int bk = 0;
    while (bk + 1 < kMaxBuckets && n < kBucketLo[bk]) bk++;
    return bk;
  };
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c2) {
    const auto& A = b->hinst[a];
    const auto& B = b->hinst[c2];
    const int ba = bucket_of(A.n), bb = bucket_of(B.n);
    if (ba != bb) return ba < bb;
    const double wa = (double)A.n * (2.0 * A.p + 30.0), wb = (double)B.n * (2.0 * B.p + 30.0);
    return wa > wb;
  });
  {
    Sched& S = b->sched;
    S = Sched();
    int pos = 0;
    for (int bk = 0; bk < kMaxBuckets; bk++) {
      S.beg[bk] = pos;
      int64_t pm = 0, fm = 0;
      while (pos < count && bucket_of(b->hinst[order[pos]].n) == bk) {
        const Inst& I = b->hinst[order[pos]];
        pm = std::max<int64_t>(pm, I.p);
        fm = std::max<int64_t>(fm, I.p * I.n);
        pos++;
      }
      S.pmax[bk] = pm;
      S.fmax[bk] = fm;
      S.threads[bk] = 256;
      S.fs[bk] = false;
      b->bucket_lo.push_back((int)kBucketLo[bk]);
    }
    S.beg[kMaxBuckets] = pos;
  }
  b->horder = order;
  Pools& P = b->P;
  std::memset(&P, 0, sizeof(P));
  P.count = count;
  const size_t N = c.size(), M = l.size();
  Inst* dinst;
  if ((st = bupload(b, &dinst, b->hinst))) return st;
  P.inst = dinst;
  std::vector<Res> rz(count);
  std::memset(rz.data(), 0, sizeof(Res) * count);
  Res* dres;
  if ((st = bupload(b, &dres, rz))) return st;
  P.res = dres;
  int* dord;
  if ((st = bupload(b, &dord, order))) return st;
  P.order = dord;
  std::vector<unsigned> hz(kMaxBuckets, 0u);
  unsigned* dh;
  if ((st = bupload(b, &dh, hz))) return st;
  P.head = dh;
  double* tmp;
  if ((st = bupload(b, &tmp, c))) return st;
  P.c = tmp;
  if ((st = bupload(b, &tmp, L))) return st;
  P.L = tmp;
  if ((st = bupload(b, &tmp, U))) return st;
  P.U = tmp;
  if ((st = bupload(b, &tmp, d))) return st;
  P.d = tmp;
  if ((st = bupload(b, &tmp, x0in))) return st;
  P.x0in = tmp;
  if ((st = bupload(b, &tmp, l))) return st;
  P.l = tmp;
  if ((st = bupload(b, &tmp, u))) return st;
  P.u = tmp;
  if ((st = bupload(b, &tmp, y0in))) return st;
  P.y0in = tmp;
  if ((st = bupload(b, &tmp, F))) return st;
  P.F = tmp;
  double** nv[] = {&P.x, &P.w, &P.Qw, &P.ATy, &P.x0, &P.w0, &P.Qw0, &P.ATy0, &P.xb, &P.wb, &P.Qwb, &P.ATyb,
                   &P.wh, &P.Qwh, &P.v, &P.zb, &P.Qxb, &P.s1, &P.s2};
  for (double** p : nv)
    if ((st = bzeros(b, p, N))) return st;
  double** mv[] = {&P.y, &P.y0, &P.yb};
  for (double** p : mv)
    if ((st = bzeros(b, p, M))) return st;
  if ((st = bzeros(b, &P.qat, (size_t)qat_total))) return st;
  if ((st = bzeros(b, &P.aqa, (size_t)aqa_total))) return st;
  int* ip;
  if ((st = bupload(b, &ip, arp))) return st;
  P.arp = ip;
  if ((st = bupload(b, &ip, aci))) return st;
  P.aci = ip;
  if ((st = bupload(b, &ip, trp))) return st;
  P.trp = ip;
  if ((st = bupload(b, &ip, tci))) return st;
  P.tci = ip;
  if ((st = bupload(b, &ip, qrp))) return st;
  P.qrp = ip;
  if ((st = bupload(b, &ip, qci))) return st;
  P.qci = ip;
  if ((st = bupload(b, &tmp, av))) return st;
  P.av = tmp;
  if ((st = bupload(b, &tmp, tv))) return st;
  P.tv = tmp;
  if ((st = bupload(b, &tmp, qv))) return st;
  P.qv = tmp;
  BCU(b, cudaStreamSynchronize(b->stream));
  BCU(b, cudaGetDevice(&b->dev));
  for (int k = 0; k < kMaxBuckets - 1; k++) {
    BCU(b, cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
    BCU(b, cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
  }
  BCU(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  b->hres.resize(count);
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_batch_create(hprqp_batch** out, int32_t count, const hprqp_problem* probs,
                                           const hprqp_params* params) {
  g_batch_err.clear();
  if (!out || count < 1 || !probs) return bfail(nullptr, HPRQP_INVALID_ARG, "need an output pointer and count >= 1");
  *out = nullptr;
  hprqp_batch* b = new hprqp_batch();
  if (params) b->prm = *params;
  else hprqp_default_params(&b->prm);
  const int bt = b->prm.batch_team;
  if (bt != 0 && bt != 64 && bt != 128 && bt != 256 && bt != 512) {
    delete b;
    return bfail(nullptr, HPRQP_INVALID_ARG, "batch_team must be 0, 64, 128, 256 or 512");
  }
  if (b->prm.check_every < 1 || b->prm.restart_every < 1) {
    delete b;
    return bfail(nullptr, HPRQP_INVALID_ARG, "check_every and restart_every must be >= 1");
  }
  if (b->prm.stream) {
    b->stream = (cudaStream_t)b->prm.stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return bfail(nullptr, HPRQP_CUDA_ERROR, "cannot create a CUDA stream (no device?)");
    }
    b->own_stream = true;
  }
  hprqp_status st = batch_create_impl(b, count, probs);
  if (st != HPRQP_OK) {
    if (g_batch_err.empty()) g_batch_err = b->err;
    brelease(b);
    return st;
  }
  *out = b;
  return HPRQP_OK;
}

// Dynamic shared memory of a block of bucket bk: its Shared state (t sized for the bucket's
// largest p) and, with the F copy, the bucket's largest F.
static bool small_p(const Sched& S, int bk) { return S.pmax[bk] <= kSmallP; }
static size_t bucket_smem(const Sched& S, int bk, bool fs) {
  return shared_bytes(small_p(S, bk)) + (fs ? (size_t)S.fmax[bk] * sizeof(double) : 0);
}

// One launch: the instances order[beg .. beg + cnt) of bucket bk with the given block size and F
// copy, at most one wave of resident blocks (each takes instances from the bucket's counter).
static cudaError_t launch_bucket(hprqp_batch* b, int bk, int beg, int cnt, int threads, bool fs, int sms,
                                 cudaStream_t s) {
  const Sched& S = b->sched;
  const KFn k = batch_kernel(fs, small_p(S, bk));
  const size_t smem = bucket_smem(S, bk, fs);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const int grid = std::max(1, std::min(cnt, sms * occ));
  k<<<grid, threads, smem, s>>>(b->P, Bucket{beg, cnt, b->P.head + bk});
  return cudaGetLastError();
}

// Whether a bucket's F copies fit a block's shared memory.
static bool fs_fits(hprqp_batch* b, int bk) {
  const Sched& S = b->sched;
  int optin = 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return S.fmax[bk] > 0 && bucket_smem(S, bk, true) <= (size_t)optin;
}

// Autotuner (row a10): per bucket of instances, time the candidate schedules on the bucket's own
// instances (the first 100 iterations of one wave of them, one launch each) and keep the one
// with the highest rate of estimated work: blocks of 512, 256, 128 or 64 threads per instance,
// each with and without a shared-memory copy of the instance's dense factor F (where every F of
// the bucket fits).  batch_team fixes the block size of every bucket (no F copy); autotune = 0 takes
// 512, 256, 128 and 64 threads from the largest n down (no F copy).
static hprqp_status batch_autotune(hprqp_batch* b, int sms) {
  Sched& S = b->sched;
  Pools& P = b->P;
  if (b->prm.batch_team || !b->prm.autotune) {
    const int fixed[kMaxBuckets] = {512, 256, 128, 64};
    for (int bk = 0; bk < kMaxBuckets; bk++) {
      S.threads[bk] = b->prm.batch_team ? b->prm.batch_team : fixed[bk];
      S.fs[bk] = false;
    }
    return HPRQP_OK;
  }
  cudaEvent_t e0, e1;
  BCU(b, cudaEventCreate(&e0));
  BCU(b, cudaEventCreate(&e1));
  const long long keep = P.max_iter;
  P.max_iter = std::min<long long>(keep, 100);
  for (int bk = 0; bk < kMaxBuckets; bk++) {
    const int cnt = S.beg[bk + 1] - S.beg[bk];
    if (cnt <= 0) continue;
    double best = 0.0;   // estimated work per millisecond of the best candidate
    for (int fs = 0; fs < 2; fs++) {
      if (fs && !fs_fits(b, bk)) continue;
      // largest blocks first; smaller ones only while they stay within 15 % of the best so far
      // (the rate falls steadily as blocks shrink past the best size)
      for (int G : {512, 256, 128, 64}) {
        // one wave: as many of the bucket's instances (largest first) as blocks of this shape fit
        // the GPU at once, so that no candidate is timed on a partial last wave; rates compare
        // the instances' estimated work (the work order's cost) per millisecond
        const KFn k = batch_kernel(fs != 0, small_p(S, bk));
        const size_t smem = bucket_smem(S, bk, fs != 0);
        int occ = 0;
        BCU(b, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BCU(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, G, smem));
        if (occ < 1) continue;   // no block of this shape fits an SM
        const int sample = std::min(cnt, sms * occ);
        double work = 0.0;
        for (int q = S.beg[bk]; q < S.beg[bk] + sample; q++) {
          const Inst& I = b->hinst[b->horder[q]];
          work += (double)I.n * (2.0 * I.p + 30.0);
        }
        BCU(b, cudaMemsetAsync(P.head + bk, 0, sizeof(unsigned), b->stream));
        BCU(b, cudaEventRecord(e0, b->stream));
        BCU(b, launch_bucket(b, bk, S.beg[bk], sample, G, fs != 0, sms, b->stream));
        BCU(b, cudaEventRecord(e1, b->stream));
        BCU(b, cudaEventSynchronize(e1));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = work / std::max(1e-3, (double)ms);
        if (b->prm.verbose >= 2)
          std::fprintf(stderr, "hprqp batch autotune: bucket %d (n >= %d): %d threads%s, %d instances: %.3f ms, "
                       "%.4g work/ms\n", bk, b->bucket_lo[bk], G, fs ? ", F in shared memory" : "", sample, ms, rate);
        if (rate > best) {
          best = rate;
          S.threads[bk] = G;
          S.fs[bk] = fs != 0;
        } else if (rate * 1.15 < best) {
          break;
        }
      }
    }
  }
  P.max_iter = keep;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_batch_solve(hprqp_batch* b, double tol, int64_t max_iter) {
  if (!b) return HPRQP_INVALID_ARG;
  b->err.clear();
  if (!(tol > 0.0) || max_iter < 1) return bfail(b, HPRQP_INVALID_ARG, "need tol > 0 and max_iter >= 1");
  BCU(b, cudaSetDevice(b->dev));
  Pools& P = b->P;
  P.tol = tol;
  P.max_iter = max_iter;
  P.alpha1 = b->prm.alpha1;
  P.alpha2 = b->prm.alpha2;
  P.alpha3 = b->prm.alpha3;
  P.alpha3_tight = b->prm.alpha3_tight;
  P.ratio_tight = b->prm.ratio_tight;
  P.power_tol = b->prm.power_tol;
  P.power_safety = b->prm.power_safety;
  P.power_max_iter = b->prm.power_max_iter;
  P.check_every = b->prm.check_every;
  P.restart_every = b->prm.restart_every;
  P.halpern_total = b->prm.halpern_total;
  P.restart_off = b->prm.restart_off;
  P.sigma_fixed = b->prm.sigma_fixed;
  P.sigma_golden = b->prm.sigma_golden;
  int sms = 0;
  BCU(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev));
  if (!b->tuned) {
    b->tuned = true;
    hprqp_status st = batch_autotune(b, sms);
    if (st != HPRQP_OK) return st;
  }
  const Sched& S = b->sched;
  auto t0 = std::chrono::steady_clock::now();
  // bucket 0 on the caller's stream, the others on side streams forked from it: each launch
  // fills the SMs its blocks fit, and the next bucket's blocks start on an SM as the previous
  // bucket's blocks leave it (largest instances first, no idle SM between buckets)
  BCU(b, cudaMemsetAsync(P.head, 0, sizeof(unsigned) * kMaxBuckets, b->stream));
  BCU(b, cudaEventRecord(b->fork, b->stream));
  b->launches = 0;
  bool joined[kMaxBuckets] = {};
  for (int bk = 0; bk < kMaxBuckets; bk++) {
    const int cnt = S.beg[bk + 1] - S.beg[bk];
    if (cnt <= 0) continue;
    cudaStream_t s = b->stream;
    if (b->launches > 0) {
      s = b->side[bk - 1];
      BCU(b, cudaStreamWaitEvent(s, b->fork, 0));
    }
    BCU(b, launch_bucket(b, bk, S.beg[bk], cnt, S.threads[bk], S.fs[bk], sms, s));
    if (s != b->stream) {
      BCU(b, cudaEventRecord(b->join[bk - 1], s));
      joined[bk] = true;
    }
    b->launches++;
  }
  for (int bk = 1; bk < kMaxBuckets; bk++)
    if (joined[bk]) BCU(b, cudaStreamWaitEvent(b->stream, b->join[bk - 1], 0));
  BCU(b, cudaMemcpyAsync(b->hres.data(), P.res, sizeof(Res) * b->count, cudaMemcpyDeviceToHost, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  b->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  b->solved = true;
  bool all = true;
  for (const Res& r : b->hres) {
    if (r.status == 3) return bfail(b, HPRQP_NUMERICAL_ERROR, "an instance hit a numerical error");
    if (r.status != 0) all = false;
  }
  return all ? HPRQP_OK : HPRQP_MAX_ITER;
}

extern "C" hprqp_status hprqp_batch_schedule(const hprqp_batch* b, int64_t* out) {
  if (!b || !out) return HPRQP_INVALID_ARG;
  for (int bk = 0; bk < kMaxBuckets; bk++) {
    int64_t* o = out + 5 * bk;
    o[0] = b->bucket_lo[bk];
    o[1] = b->sched.beg[bk + 1] - b->sched.beg[bk];
    o[2] = b->sched.threads[bk];
    o[3] = b->sched.fs[bk] ? 1 : 0;
    o[4] = b->sched.fs[bk] ? b->sched.fmax[bk] : 0;
  }
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_batch_get(hprqp_batch* b, int32_t i, double* x, double* y, double* z, hprqp_kkt* kkt) {
  if (!b) return HPRQP_INVALID_ARG;
  if (!b->solved) return bfail(b, HPRQP_INVALID_ARG, "hprqp_batch_get before hprqp_batch_solve");
  if (i < 0 || i >= b->count) return bfail(b, HPRQP_INVALID_ARG, "instance index out of range");
  const Inst& I = b->hinst[i];
  if (x) BCU(b, cudaMemcpyAsync(x, b->P.xb + I.on, I.n * sizeof(double), cudaMemcpyDefault, b->stream));
  if (y && I.m) BCU(b, cudaMemcpyAsync(y, b->P.yb + I.om, I.m * sizeof(double), cudaMemcpyDefault, b->stream));
  if (z) BCU(b, cudaMemcpyAsync(z, b->P.zb + I.on, I.n * sizeof(double), cudaMemcpyDefault, b->stream));
  BCU(b, cudaStreamSynchronize(b->stream));
  if (kkt) {
    const Res& r = b->hres[i];
    std::memset(kkt, 0, sizeof(*kkt));
    kkt->eta_p = r.eta_p;
    kkt->eta_d = r.eta_d;
    kkt->eta_gap = r.eta_gap;
    kkt->rel_kkt = std::max(r.eta_p, std::max(r.eta_d, r.eta_gap));
    kkt->pobj = r.pobj;
    kkt->dobj = r.dobj;
    kkt->iters = r.iters;
    kkt->restarts = r.restarts;
    kkt->sigma = r.sigma;
    kkt->lambda_A = r.lamA;
    kkt->lambda_Q = r.lamQ;
    kkt->solve_seconds = b->seconds;
    kkt->kernel_launches = b->launches;
    kkt->status = r.status;
  }
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_batch_stats(hprqp_batch* b, double* seconds, int64_t* kernel_launches) {
  if (!b) return HPRQP_INVALID_ARG;
  if (seconds) *seconds = b->seconds;
  if (kernel_launches) *kernel_launches = b->launches;
  return HPRQP_OK;
}

extern "C" void hprqp_batch_destroy(hprqp_batch* b) { brelease(b); }

extern "C" const char* hprqp_batch_last_error(const hprqp_batch* b) {
  return b ? b->err.c_str() : g_batch_err.c_str();
}
