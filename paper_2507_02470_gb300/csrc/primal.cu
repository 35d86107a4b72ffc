// Primal HPR methods of Appendix A (Algorithms 6 and 7), for ablation against Algorithm 4.
//
// Both run on the reformulations with the slack s = Ax (and v = x for Algorithm 7), with the
// proximal terms that make every step explicit, fixed sigma and the Halpern step of Step 5
// without restarts, as printed.  The products A x, A^T w and Q x run on the solver's own
// operator kernels (launch_apply); the elementwise steps and the stopping rule of Sec. 4.1 are
// the kernels below.
//
//   Steps 1-2   q = Ax - y/sigma, sbar = Pi_K(q), ybar = sigma (Pi_K(q) - q) (= y + sigma (sbar
//               - Ax), in the form whose sign matches K exactly), w = 2 ybar - y
//   Alg. 7      vbar = (lambda_Q v - Qv + sigma x - t) / (lambda_Q + sigma), tbar = t + sigma (vbar - x)
//   Step 3      r = x - g / tau, xbar = Prox_{phi/tau}(r), zbar = tau (xbar - r), with
//               Alg. 6: g = Qx + c - A^T w,                            tau = lambda_Q + sigma lambda_A
//               Alg. 7: g = c - A^T w - tbar + sigma (x - vbar),       tau = sigma (1 + lambda_A)
//   Steps 4-5   u = (u^0 + (k+1)(2 ubar - u)) / (k+2) for u = (x, s, y) (and v, t)
#include <cmath>

#include "kernels.cuh"

namespace hprqp {
namespace {

__global__ void k_p_rows(const double* __restrict__ Ax, const double* __restrict__ y, const double* __restrict__ l,
                         const double* __restrict__ u, double sigma, double inv_sigma, int64_t m,
                         double* __restrict__ sb, double* __restrict__ yb, double* __restrict__ w) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    const double q = Ax[i] - y[i] * inv_sigma;
    const double s = iclamp(q, l[i], u[i]);
    const double ybar = sigma * (s - q);
    sb[i] = s;
    yb[i] = ybar;
    w[i] = 2.0 * ybar - y[i];
  }
}

__global__ void k_p_vt(const double* __restrict__ v, const double* __restrict__ Qv, const double* __restrict__ x,
                       const double* __restrict__ t, double lamQ, double sigma, int64_t n, double* __restrict__ vb,
                       double* __restrict__ tb) {
  const double inv = 1.0 / (lamQ + sigma);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
    const double vv = (lamQ * v[j] - Qv[j] + sigma * x[j] - t[j]) * inv;
    vb[j] = vv;
    tb[j] = t[j] + sigma * (vv - x[j]);
  }
}

__global__ void k_p_x(const double* __restrict__ x, const double* __restrict__ Qv, const double* __restrict__ c,
                      const double* __restrict__ ATw, const double* __restrict__ vb, const double* __restrict__ tb,
                      const double* __restrict__ L, const double* __restrict__ U, int phi, double lambda, double sigma,
                      double tau, int two, int64_t n, double* __restrict__ xb, double* __restrict__ zb) {
  const double inv_tau = 1.0 / tau;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
    const double g = two ? c[j] - ATw[j] - tb[j] + sigma * (x[j] - vb[j]) : Qv[j] + c[j] - ATw[j];
    const double r = x[j] - g * inv_tau;
    const double xv = prox_phi(phi, r, L[j], U[j], lambda * inv_tau);
    xb[j] = xv;
    zb[j] = tau * (xv - r);
  }
}

// u = a u0 + b (2 ubar - u) for up to three vector triples of length len
struct Halp {
  double* u[3];
  const double* u0[3];
  const double* ub[3];
  int count;
};
__global__ void k_p_halpern(Halp H, double a, double b, int64_t len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < len; j += stride)
    for (int q = 0; q < H.count; q++) H.u[q][j] = a * H.u0[q][j] + b * (2.0 * H.ub[q][j] - H.u[q][j]);
}

// ---- the stopping rule of Sec. 4.1 at (xbar, ybar, zbar): per-block partials, then one block
constexpr int kPN = 8;   // n-terms: max rd, max|A^T y|, max|Qx|, x.Qx, c.x, |x|_1, phi*(-z), (unused)
constexpr int kPM = 4;   // m-terms: max|Ax - Pi(Ax)|, max|Ax|, -delta*_K(-y), (unused)

__global__ void __launch_bounds__(kThreads) k_p_eta_n(const double* __restrict__ xb, const double* __restrict__ Qxb,
                                                      const double* __restrict__ ATyb, const double* __restrict__ zb,
                                                      const double* __restrict__ c, const double* __restrict__ L,
                                                      const double* __restrict__ U, int phi, double lambda,
                                                      int64_t n, double* __restrict__ part) {
  __shared__ double red[kPN * 32];
  double t[kPN] = {0, 0, 0, 0, 0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
    const double x = xb[j], qx = Qxb[j], aty = ATyb[j];
    t[0] = imax(t[0], iabs(aty - qx + zb[j] - c[j]));
    t[1] = imax(t[1], iabs(aty));
    t[2] = imax(t[2], iabs(qx));
    t[3] = fma(x, qx, t[3]);
    t[4] = fma(c[j], x, t[4]);
    if (phi != PHI_BOX) t[5] += iabs(x);
    t[6] += conj_phi_term(phi, zb[j], L[j], U[j], lambda);
  }
  block_reduce<kPN>(t, 0x7u, red);   // terms 0-2 are maxima
  if (threadIdx.x == 0)
    for (int i = 0; i < kPN; i++) part[(size_t)blockIdx.x * kPN + i] = t[i];
}

__global__ void __launch_bounds__(kThreads) k_p_eta_m(const double* __restrict__ Axb, const double* __restrict__ yb,
                                                      const double* __restrict__ l, const double* __restrict__ u,
                                                      int64_t m, double* __restrict__ part) {
  __shared__ double red[kPM * 32];
  double t[kPM] = {0, 0, 0, 0};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    const double ax = Axb[i], lo = l[i], hi = u[i], y = yb[i];
    t[0] = imax(t[0], iabs(ax - iclamp(ax, lo, hi)));
    t[1] = imax(t[1], iabs(ax));
    if (igt0(y)) t[2] += lo * y;
    else if (ilt0(y)) t[2] += hi * y;
  }
  block_reduce<kPM>(t, 0x3u, red);
  if (threadIdx.x == 0)
    for (int i = 0; i < kPM; i++) part[(size_t)blockIdx.x * kPM + i] = t[i];
}

// out: eta_p, eta_d, eta_gap, pobj, dobj
__global__ void __launch_bounds__(kThreads) k_p_eta_fin(const double* __restrict__ pn, int nbn,
                                                        const double* __restrict__ pm, int nbm, double b_inf,
                                                        double c_inf, int phi, double lambda, double* __restrict__ out) {
  __shared__ double red[kPN * 32];
  double tn[kPN], tm[kPM];
  reduce_partials<kPN>(pn, nbn, kPN, 0x7u, tn, red);
  __syncthreads();
  for (int i = 0; i < kPM; i++) tm[i] = 0.0;
  if (nbm > 0) reduce_partials<kPM>(pm, nbm, kPM, 0x3u, tm, red);
  if (threadIdx.x == 0) {
    const double eta_p = tm[0] / (1.0 + fmax(b_inf, tm[1]));
    const double eta_d = tn[0] / (1.0 + fmax(c_inf, fmax(tn[1], tn[2])));
    const double pobj = 0.5 * tn[3] + tn[4] + (phi != PHI_BOX ? lambda * tn[5] : 0.0);
    const double dobj = -0.5 * tn[3] + tm[2] - tn[6];
    out[0] = eta_p;
    out[1] = eta_d;
    out[2] = fabs(pobj - dobj) / (1.0 + fmax(fabs(pobj), fabs(dobj)));
    out[3] = pobj;
    out[4] = dobj;
  }
}

int blocks_for(int64_t len) { return (int)std::max<int64_t>(1, std::min<int64_t>((len + kThreads - 1) / kThreads, 152 * 8)); }

}  // namespace

cudaError_t primal_rows(const double* Ax, const double* y, const double* l, const double* u, double sigma, int64_t m,
                        double* sb, double* yb, double* w, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  k_p_rows<<<blocks_for(m), kThreads, 0, s>>>(Ax, y, l, u, sigma, 1.0 / sigma, m, sb, yb, w);
  return cudaGetLastError();
}

cudaError_t primal_vt(const double* v, const double* Qv, const double* x, const double* t, double lamQ, double sigma,
                      int64_t n, double* vb, double* tb, cudaStream_t s) {
  k_p_vt<<<blocks_for(n), kThreads, 0, s>>>(v, Qv, x, t, lamQ, sigma, n, vb, tb);
  return cudaGetLastError();
}

cudaError_t primal_x(const double* x, const double* Qv, const double* c, const double* ATw, const double* vb,
                     const double* tb, const double* L, const double* U, int phi, double lambda, double sigma,
                     double tau, int two, int64_t n, double* xb, double* zb, cudaStream_t s) {
  k_p_x<<<blocks_for(n), kThreads, 0, s>>>(x, Qv, c, ATw, vb, tb, L, U, phi, lambda, sigma, tau, two, n, xb, zb);
  return cudaGetLastError();
}

cudaError_t primal_halpern(double* const* u, const double* const* u0, const double* const* ub, int count, double a,
                           double b, int64_t len, cudaStream_t s) {
  if (len <= 0 || count <= 0) return cudaSuccess;
  Halp H;
  H.count = count;
  for (int q = 0; q < 3; q++) {
    H.u[q] = q < count ? u[q] : nullptr;
    H.u0[q] = q < count ? u0[q] : nullptr;
    H.ub[q] = q < count ? ub[q] : nullptr;
  }
  k_p_halpern<<<blocks_for(len), kThreads, 0, s>>>(H, a, b, len);
  return cudaGetLastError();
}

int primal_eta_blocks(int64_t len) { return blocks_for(len); }

cudaError_t primal_eta(const double* xb, const double* Qxb, const double* ATyb, const double* zb, const double* Axb,
                       const double* yb, const Args& a, double b_inf, double c_inf, double lambda, double* part_n,
                       double* part_m, double* out, cudaStream_t s) {
  const Vec& V = a.V;
  const int nbn = blocks_for(a.n), nbm = a.m > 0 ? blocks_for(a.m) : 0;
  k_p_eta_n<<<nbn, kThreads, 0, s>>>(xb, Qxb, ATyb, zb, V.c, V.L, V.U, a.phi, lambda, a.n, part_n);
  if (nbm) k_p_eta_m<<<nbm, kThreads, 0, s>>>(Axb, yb, V.l, V.u, a.m, part_m);
  k_p_eta_fin<<<1, kThreads, 0, s>>>(part_n, nbn, part_m, nbm, b_inf, c_inf, a.phi, lambda, out);
  return cudaGetLastError();
}

}  // namespace hprqp
