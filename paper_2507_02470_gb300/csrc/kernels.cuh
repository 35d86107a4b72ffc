// Device code of one inner step of HPR-QP (arXiv 2507.02470, Algorithm 4), for one instance.
//
// One inner step is five fused passes; the Sec. 3.1 updates run in the prologues and
// epilogues of the operator products, so each vector element crosses HBM once per pass:
//   K1  elementwise n: pending Halpern / restart update of (x, w_Q, Qw, A^*y), then
//       eqs. (3.1)-(3.3): r_z, xbar = Prox(r_z), zbar, what = 2 xbar - x, wbar_{1/2}
//   K2  Q wbar_{1/2} (+ Q xbar on stopping tests); epilogue v = what + sigma (Qw - Q wbar_{1/2})
//   K3  A v (+ A xbar); prologue Halpern on y; epilogue eq. (3.5): ybar = (Pi_K(r_y) - r_y)/(sigma lA)
//   K4  A^T ybar; epilogue eq. (3.3): wbar = wbar_{1/2} + sigma/(1+sigma lQ) (A^* ybar - A^* y)
//   K5  Q wbar; epilogue: R~ terms of the metric (2.12) and the Sec. 4.1 residuals; the last
//       block to finish runs the controller (restart rules (3.6)-(3.8), termination) and
//       selects the variant of the next step.
// The images Q w and A^* y of the Halpern iterate follow the Halpern recurrence (both maps
// are linear), so only wbar_{1/2}, v, ybar and wbar meet an operator each step.  Restarts
// run one more pass for theta~ of eq. (3.11) and Algorithm 5.
//
// Variants (template VAR): 0 plain step, 1 step that evaluates R~, 2 step that evaluates the
// stopping rule (R~ as flagged at run time), 3 everything decided at run time.  The plain
// variant carries none of the reduction code, which keeps its register count and latency low.
#pragma once
#include <cuda_runtime.h>

#include "solver.cuh"

// Loads of vectors that other blocks wrote.  Separate launches may read them through the
// read-only cache and with restrict-qualified pointers; the persistent solver, which runs
// every pass inside one launch separated by grid barriers, compiles these bodies with
// HPRQP_COHERENT so that such loads go to L2 (__ldcg, see gather_f64) and no pointer claims
// read-only data.
#ifdef HPRQP_COHERENT
#define HPRQP_RESTRICT
#else
#define HPRQP_RESTRICT __restrict__
#endif

namespace hprqp {

// L2 eviction priorities for the CSR passes: the stored matrix is read once per pass
// (evict first, no L1 allocation) while the gathered vector is reused by every row that names
// its entries (evict last), so the 4-8 MB vectors stay in L2 while 36 MB of A streams by.
// The persistent solver keeps plain coherent loads.
#ifdef HPRQP_COHERENT
struct L2Pol {
  __device__ __forceinline__ L2Pol() {}
};
__device__ __forceinline__ double gather_f64(const double* p, const L2Pol&) { return __ldcg(p); }
__device__ __forceinline__ double stream_f64(const double* p, const L2Pol&) { return *p; }
__device__ __forceinline__ int stream_i32(const int* p, const L2Pol&) { return *p; }
#else
struct L2Pol {
  unsigned long long keep, drop;
  __device__ __forceinline__ L2Pol() {
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(drop));
  }
};
__device__ __forceinline__ double gather_f64(const double* p, const L2Pol& q) {
  double v;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(q.keep));
  return v;
}
__device__ __forceinline__ double stream_f64(const double* p, const L2Pol& q) {
  double v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(q.drop));
  return v;
}
__device__ __forceinline__ int stream_i32(const int* p, const L2Pol& q) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(q.drop));
  return v;
}
#endif

// The value a CSR pass multiplies entry (i, c) with: the c-th element of a vector in memory, or,
// for a thin factor term B (see QDev::inl), (B x)_c formed from row c of B on demand (entries
// in stored order), so that the pass needs no pre-pass writing t = B x first.
struct GatherX {
  const double* p;
  __device__ __forceinline__ double operator()(int c, const L2Pol& pol) const { return gather_f64(p + c, pol); }
};
struct FacRowX {
  const int* rp;
  const int* ci;
  const double* v;
  const double* x;
  __device__ __forceinline__ double operator()(int c, const L2Pol& pol) const {
    const int b = rp[c], e = rp[c + 1];
    double s = 0.0;
    for (int k = b; k < e; k++) s = fma(v[k], gather_f64(x + ci[k], pol), s);
    return s;
  }
};

template <class X>
constexpr bool kOnDemand = false;
template <>
constexpr bool kOnDemand<FacRowX> = true;

// Conditional-node handles set by the controller (graph mode); zero flags when unused.
struct Handles {
  unsigned long long sw_next = 0;   // SWITCH node of the next inner step
  unsigned long long rs_cur = 0;    // IF node of this step's restart pass
  int has_next = 0, has_rs = 0;
  int fixed = 0;                    // 1: graph with a fixed variant schedule (values of fixed_value)
};

// Entry of every kernel that the step launchers may start as a programmatic dependent launch:
// wait until the preceding kernel of the stream has finished and its writes are visible (a
// no-op after an ordinary launch), then allow the next kernel to begin launching.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

enum { VAR_PLAIN = 0, VAR_R = 1, VAR_T = 2, VAR_RUNTIME = 3 };

template <int VAR>
__device__ __forceinline__ bool var_rtest(const Ctrl* C) {
  return VAR == VAR_PLAIN ? false : VAR == VAR_R ? true : (bool)C->rtest;
}
template <int VAR>
__device__ __forceinline__ bool var_ttest(const Ctrl* C) {
  return VAR == VAR_PLAIN || VAR == VAR_R ? false : VAR == VAR_T ? true : (bool)C->ttest;
}

// switch value of the next step: 0 plain, 1 R~ test, 2 stopping test, 3 nothing (done)
__device__ __forceinline__ unsigned next_variant(const Ctrl& C) {
  return C.done ? 3u : C.ttest ? 2u : C.rtest ? 1u : 0u;
}
// switch value in the fixed-schedule graph, at a step that follows a possible restart:
// 0 the step's scheduled variant, 1 with the R~ test (first step after a restart), 2 the
// restart pass of Algorithm 5 and then that step, 3 nothing (done)
__device__ __forceinline__ unsigned fixed_value(const Ctrl& C) {
  return C.done ? 3u : C.restart_pending ? 2u : C.rtest ? 1u : 0u;
}
__device__ __forceinline__ unsigned switch_value(const Ctrl& C, const Handles& hd) {
  return hd.fixed ? fixed_value(C) : next_variant(C);
}

// ------------------------------------------------------------------------------------ prox
__device__ __forceinline__ double prox_phi(int phi, double r, double L, double U, double tau) {
  if (phi == PHI_BOX) return iclamp(r, L, U);
  const double s = r - iclamp(r, -tau, tau);  // soft threshold
  if (phi == PHI_L1) return s;
  return iclamp(s, L, U);
}

// phi^*(-z) contribution of one coordinate (0 * inf = 0 for the box).  For lam|x| + the box,
// sup over [L, U] of (-z x - lam |x|): a finite end point or 0, given z <= lam where L = -inf
// and z >= -lam where U = +inf.  zbar from the prox (eq. (3.1)) meets that in exact
// arithmetic but can cross the edge by rounding, so on an infinite side a z within 64 ulps of
// the edge (relative to max(1, lam)) is put on the edge (the pure l1 term, 0 on [-lam, lam],
// makes the same assumption); a z further out is outside the domain and gives +inf.
__device__ __forceinline__ double conj_phi_term(int phi, double z, double L, double U, double lam) {
  if (phi == PHI_L1) return 0.0;
  if (phi == PHI_BOX) {
    double t = 0.0;
    if (igt0(z)) t = -L * z;
    else if (ilt0(z)) t = -U * z;
    return t;
  }
  const double edge = 64.0 * 2.220446049250313e-16 * fmax(1.0, lam);
  if (iisinf(L) && z > lam) {
    if (z - lam > edge) return INFINITY;
    z = lam;
  }
  if (iisinf(U) && z < -lam) {
    if (-lam - z > edge) return INFINITY;
    z = -lam;
  }
  double best = -INFINITY;
  if (!iisinf(L)) best = imax(best, -z * L - lam * iabs(L));
  if (!iisinf(U)) best = imax(best, -z * U - lam * iabs(U));
  if (L <= 0.0 && U >= 0.0) best = imax(best, 0.0);
  return best;
}

// ------------------------------------------------------------------------------------ CSR pass
// Row sums of a chunk of kChunk rows, G lanes per row, into shared rs0/rs1 (add: accumulate).
template <int G, int NR, class X0, class X1>
__device__ __forceinline__ void csr_chunk_lanes(const Csr& M, int64_t row0, const X0& x0, const X1& x1, double* rs0,
                                                double* rs1, bool add) {
  const int lane = threadIdx.x % G;
  const int grp = threadIdx.x / G;
  constexpr int NG = kThreads / G;
  const L2Pol pol;
#pragma unroll 1
  for (int rr = grp; rr < kChunk; rr += NG) {
    const int64_t row = row0 + rr;
    double s0 = 0.0, s1 = 0.0;
    if (row < M.rows && kOnDemand<X0>) {
      // values formed on demand (thin factor): rows of B^T hold a few entries at most, so one
      // entry at a time, with no unrolled loads to keep in registers
      const int b = stream_i32(M.rp + row, pol), e = stream_i32(M.rp + row + 1, pol);
      for (int k = b + lane; k < e; k += G) {
        const int c = stream_i32(M.ci + k, pol);
        const double v = stream_f64(M.v + k, pol);
        s0 = fma(v, x0(c, pol), s0);
        if (NR == 2) s1 = fma(v, x1(c, pol), s1);
      }
    } else if (row < M.rows) {
      const int b = stream_i32(M.rp + row, pol), e = stream_i32(M.rp + row + 1, pol);
      int k = b + lane;
      for (; k + 3 * G < e; k += 4 * G) {
        const int c0 = stream_i32(M.ci + k, pol), c1 = stream_i32(M.ci + k + G, pol),
                  c2 = stream_i32(M.ci + k + 2 * G, pol), c3 = stream_i32(M.ci + k + 3 * G, pol);
        const double v0 = stream_f64(M.v + k, pol), v1 = stream_f64(M.v + k + G, pol),
                     v2 = stream_f64(M.v + k + 2 * G, pol), v3 = stream_f64(M.v + k + 3 * G, pol);
        const double a0 = x0(c0, pol), a1 = x0(c1, pol), a2 = x0(c2, pol), a3 = x0(c3, pol);
        s0 = fma(v0, a0, s0);
        s0 = fma(v1, a1, s0);
        s0 = fma(v2, a2, s0);
        s0 = fma(v3, a3, s0);
        if (NR == 2) {
          const double b0 = x1(c0, pol), b1 = x1(c1, pol), b2 = x1(c2, pol), b3 = x1(c3, pol);
          s1 = fma(v0, b0, s1);
          s1 = fma(v1, b1, s1);
          s1 = fma(v2, b2, s1);
          s1 = fma(v3, b3, s1);
        }
      }
      // the remaining 0-3 entries of this lane: all loads issued before the accumulation,
      // which keeps the entry order (and so the sums) of the one-at-a-time loop
      if (k < e) {
        const bool h1 = k + G < e, h2 = k + 2 * G < e;
        const int c0 = stream_i32(M.ci + k, pol);
        const int c1 = h1 ? stream_i32(M.ci + k + G, pol) : c0;
        const int c2 = h2 ? stream_i32(M.ci + k + 2 * G, pol) : c0;
        const double v0 = stream_f64(M.v + k, pol);
        const double v1 = h1 ? stream_f64(M.v + k + G, pol) : 0.0;
        const double v2 = h2 ? stream_f64(M.v + k + 2 * G, pol) : 0.0;
        const double a0 = x0(c0, pol);
        const double a1 = h1 ? x0(c1, pol) : 0.0;
        const double a2 = h2 ? x0(c2, pol) : 0.0;
        s0 = fma(v0, a0, s0);
        if (h1) s0 = fma(v1, a1, s0);
        if (h2) s0 = fma(v2, a2, s0);
        if (NR == 2) {
          const double b0 = x1(c0, pol);
          const double b1 = h1 ? x1(c1, pol) : 0.0;
          const double b2 = h2 ? x1(c2, pol) : 0.0;
          s1 = fma(v0, b0, s1);
          if (h1) s1 = fma(v1, b1, s1);
          if (h2) s1 = fma(v2, b2, s1);
        }
      }
    }
    if (G > 1) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o, G);
        if (NR == 2) s1 += __shfl_down_sync(0xffffffffu, s1, o, G);
      }
    }
    if (lane == 0 && row < M.rows) {
      rs0[rr] = add ? rs0[rr] + s0 : s0;
      if (NR == 2) rs1[rr] = add ? rs1[rr] + s1 : s1;
    }
  }
}

// Staged form of the same row sums (G = 0).  A chunk's entries [rp[row0], rp[row0 + R]) form
// one contiguous range, which the whole block streams in windows of kWin entries (coalesced
// index and value loads, every gather of a window in flight at once) into shared memory; each
// thread then sums its own row's entries of the window in entry order.  Rows of a few tens of
// entries are latency-bound in the lane form, which walks index -> gather row after row; here
// one such round trip serves up to kWin entries of many rows.
constexpr int kWin = 1024;
template <int NR, class X0, class X1>
__device__ __forceinline__ void csr_chunk_staged(const Csr& M, int64_t row0, const X0& x0, const X1& x1, double* rs0,
                                                 double* rs1, bool add) {
  __shared__ int srp[kChunk + 1];
  __shared__ double sv[kWin];
  __shared__ double sx[NR][kWin];
  constexpr int kPer = kWin / kThreads;
  const int t = threadIdx.x;
  const L2Pol pol;
  const int nr = (int)(M.rows - row0 < (int64_t)kChunk ? M.rows - row0 : (int64_t)kChunk);
  if (nr <= 0) return;   // block-uniform: no row of this matrix in the chunk
  __syncthreads();   // an earlier pass over this chunk may still read srp, sv, sx
  for (int i = t; i <= nr; i += kThreads) srp[i] = stream_i32(M.rp + row0 + i, pol);
  __syncthreads();
  const int b = srp[0], e = srp[nr];
  const int rb = t < nr ? srp[t] : 0, re = t < nr ? srp[t + 1] : 0;
  double s0 = 0.0, s1 = 0.0;
#pragma unroll 1
  for (int w0 = b; w0 < e; w0 += kWin) {
    const int wn = e - w0 < kWin ? e - w0 : kWin;
    int c[kPer];
    double v[kPer], g0[kPer], g1[kPer];
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      const int i = t + q * kThreads;
      c[q] = i < wn ? stream_i32(M.ci + w0 + i, pol) : 0;
      v[q] = i < wn ? stream_f64(M.v + w0 + i, pol) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      const int i = t + q * kThreads;
      g0[q] = i < wn ? x0(c[q], pol) : 0.0;
      if (NR == 2) g1[q] = i < wn ? x1(c[q], pol) : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kPer; q++) {
      const int i = t + q * kThreads;
      if (i < wn) {
        sv[i] = v[q];
        sx[0][i] = g0[q];
        if (NR == 2) sx[NR - 1][i] = g1[q];
      }
    }
    __syncthreads();
    const int lo = (rb > w0 ? rb : w0) - w0, hi = (re < w0 + wn ? re : w0 + wn) - w0;
    for (int k = lo; k < hi; k++) {
      s0 = fma(sv[k], sx[0][k], s0);
      if (NR == 2) s1 = fma(sv[k], sx[NR - 1][k], s1);
    }
    __syncthreads();
  }
  if (t < nr) {
    rs0[t] = add ? rs0[t] + s0 : s0;
    if (NR == 2) rs1[t] = add ? rs1[t] + s1 : s1;
  }
}

// SELL form of the same row sums (G = -1, matrices with a SELL copy): warp w of the block takes
// slice row0 / 32 + w, each lane one row of it, so every load of indices and values is
// coalesced and every FMA works on 32 rows.
template <int NR, class X0, class X1>
__device__ __forceinline__ void csr_chunk_sell(const Csr& M, int64_t row0, const X0& x0, const X1& x1, double* rs0,
                                               double* rs1, bool add) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t sl = row0 / 32 + warp;
  if (sl * 32 >= M.rows) return;   // the same for the whole warp
  const L2Pol pol;
  const int r = M.sperm[sl * 32 + lane];
  const int b = M.soff[sl], e = M.soff[sl + 1];
  double s0 = 0.0, s1 = 0.0;
  int q = b + lane;
  for (; q + 3 * 32 < e; q += 4 * 32) {
    const int c0 = stream_i32(M.sci + q, pol), c1 = stream_i32(M.sci + q + 32, pol),
              c2 = stream_i32(M.sci + q + 64, pol), c3 = stream_i32(M.sci + q + 96, pol);
    const double v0 = stream_f64(M.sv + q, pol), v1 = stream_f64(M.sv + q + 32, pol),
                 v2 = stream_f64(M.sv + q + 64, pol), v3 = stream_f64(M.sv + q + 96, pol);
    const double a0 = x0(c0, pol), a1 = x0(c1, pol), a2 = x0(c2, pol), a3 = x0(c3, pol);
    s0 = fma(v0, a0, s0);
    s0 = fma(v1, a1, s0);
    s0 = fma(v2, a2, s0);
    s0 = fma(v3, a3, s0);
    if (NR == 2) {
      const double b0 = x1(c0, pol), b1 = x1(c1, pol), b2 = x1(c2, pol), b3 = x1(c3, pol);
      s1 = fma(v0, b0, s1);
      s1 = fma(v1, b1, s1);
      s1 = fma(v2, b2, s1);
      s1 = fma(v3, b3, s1);
    }
  }
  for (; q < e; q += 32) {
    const int c = stream_i32(M.sci + q, pol);
    const double v = stream_f64(M.sv + q, pol);
    s0 = fma(v, x0(c, pol), s0);
    if (NR == 2) s1 = fma(v, x1(c, pol), s1);
  }
  if (r >= 0) {
    rs0[r - row0] = add ? rs0[r - row0] + s0 : s0;
    if (NR == 2) rs1[r - row0] = add ? rs1[r - row0] + s1 : s1;
  }
}

// Row sums of a chunk in the schedule G; a matrix without a SELL copy takes one lane per row
// where G asks for the SELL form.
template <int G, int NR, class X0, class X1>
__device__ __forceinline__ void csr_chunk_x(const Csr& M, int64_t row0, const X0& x0, const X1& x1, double* rs0,
                                            double* rs1, bool add) {
  if constexpr (G == 0) {
    csr_chunk_staged<NR>(M, row0, x0, x1, rs0, rs1, add);
  } else if constexpr (G == -1) {
    if (M.soff) csr_chunk_sell<NR>(M, row0, x0, x1, rs0, rs1, add);
    else csr_chunk_lanes<1, NR>(M, row0, x0, x1, rs0, rs1, add);
  } else {
    csr_chunk_lanes<G, NR>(M, row0, x0, x1, rs0, rs1, add);
  }
}
template <int G, int NR>
__device__ __forceinline__ void csr_chunk(const Csr& M, int64_t row0, const double* HPRQP_RESTRICT x0,
                                          const double* HPRQP_RESTRICT x1, double* rs0, double* rs1, bool add) {
  csr_chunk_x<G, NR>(M, row0, GatherX{x0}, GatherX{x1}, rs0, rs1, add);
}

// All CSR-like parts of Q (explicit CSR and every B_f^T with its intermediate t_f) for a chunk.
// inl: the pass belongs to an inner step, where a thin factor term (Q.inl) forms t_f = B_f x on
// demand from B_f's rows (x = x0, and x1 for the second vector) instead of reading t.
template <int G, int NR>
__device__ __forceinline__ void q_csr_chunk(const QDev& Q, int64_t row0, const double* x0, const double* x1,
                                            const double* t0, const double* t1, double* rs0, double* rs1,
                                            bool inl = false) {
  bool add = false;
  if (Q.csr.rows) {
    csr_chunk<G, NR>(Q.csr, row0, x0, x1, rs0, rs1, false);
    add = true;
  }
  for (int f = 0; f < Q.nfac; f++) {
    if (NR == 1 && Q.tiled[f]) continue;   // B_f^T t_f formed by the tiled kernels (q_local)
    if (inl && Q.inl[f]) {
      const Csr& B = Q.fac[f];
      csr_chunk_x<G, NR>(Q.fact[f], row0, FacRowX{B.rp, B.ci, B.v, x0}, FacRowX{B.rp, B.ci, B.v, x1}, rs0, rs1, add);
    } else {
      csr_chunk<G, NR>(Q.fact[f], row0, t0 + Q.toff[f], NR == 2 ? t1 + Q.toff[f] : nullptr, rs0, rs1, add);
    }
    add = true;
  }
  if (!add) {
    for (int rr = threadIdx.x; rr < kChunk; rr += kThreads) {
      rs0[rr] = 0.0;
      if (NR == 2) rs1[rr] = 0.0;
    }
  }
}

// Row-local parts of (Q x)_j: diagonal, symmetric band, F_g^T t_g of the dense factors, and
// (tiled_u: a one-vector pass) the tiled factors' B_f^T t_f formed before the pass.
__device__ __forceinline__ double q_local(const QDev& Q, int64_t j, const double* HPRQP_RESTRICT x,
                                          const double* HPRQP_RESTRICT t, bool with_dense, bool tiled_u) {
  double acc = 0.0;
  if (Q.diag) acc = Q.diag[j] * x[j];
  if (Q.ndia) {
    // diagonals stored by increasing offset: the main diagonal, if present, is the first
    int k = 0;
    if (Q.dia_off[0] == 0) {
      acc = fma(Q.dia[j], x[j], acc);
      k = 1;
    }
    for (; k < Q.ndia; k++) {
      const int o = Q.dia_off[k];
      const double* d = Q.dia + (size_t)k * Q.n;
      // entries past either end of the band contribute 0: the operands are selected rather than
      // the FMAs predicated, so every lane of the warp issues the same two FMAs
      const bool up = j + o < Q.n, dn = j - o >= 0;
      const double du = up ? d[j] : 0.0, xu = up ? x[j + o] : 0.0;
      const double dd = dn ? d[j - o] : 0.0, xd = dn ? x[j - o] : 0.0;
      acc = fma(du, xu, acc);
      acc = fma(dd, xd, acc);
    }
  }
  if (Q.qap_d) acc += t[Q.qap_off + j];   // (Q_qap x)_j, formed before the pass
  if (tiled_u)
    for (int f = 0; f < Q.nfac; f++)
      if (Q.tiled[f]) acc += t[Q.uoff[f] + j];
  if (with_dense) {
    for (int g = 0; g < Q.ndense; g++) {
      const double* F = Q.dense[g];
      const double* tg = t + Q.toff[Q.nfac + g];
      const int64_t p = Q.dense_p[g];
      for (int64_t r = 0; r < p; r++) acc = fma(F[(size_t)r * Q.n + j], tg[r], acc);
    }
  }
  return acc;
}

// ------------------------------------------------------------------------------------ K1
template <int VAR>
__device__ __forceinline__ void zx_body(const Args& a) {
  const Ctrl* HPRQP_RESTRICT C = a.C;
  if (C->done) return;
  const int mode = C->mode;
  const double ha = C->ha, hb = C->hb, sigma = C->sigma, c1 = C->c1, c2 = C->c2, tau = C->tau,
               inv_sigma = C->inv_sigma;
  const bool ttest = var_ttest<VAR>(C);
  const bool HQ = a.Q.present(), HA = a.m > 0;
  const int phi = a.phi;
  const Vec& V = a.V;
  // with m = 0 the y-step is absent and wbar = wbar_{1/2}: write it straight to wb;
  // with Q = 0, v = what (K2 is skipped)
  double* whout = HA ? V.wh : V.wb;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n; j += stride) {
    double x, w = 0.0, qw = 0.0, aty = 0.0;
    if (mode == 1) {
      // Halpern: u = 1/(i+2) u^{r,0} + (i+1)/(i+2) (2 ubar - u)
      x = fma(hb, fma(2.0, V.xb[j], -V.x[j]), ha * V.x0[j]);
      V.x[j] = x;
      if (HQ) {
        w = fma(hb, fma(2.0, V.wb[j], -V.w[j]), ha * V.w0[j]);
        qw = fma(hb, fma(2.0, V.Qwb[j], -V.Qw[j]), ha * V.Qw0[j]);
        V.w[j] = w;
        V.Qw[j] = qw;
      }
      if (HA) {
        aty = fma(hb, fma(2.0, V.ATyb[j], -V.ATy[j]), ha * V.ATy0[j]);
        V.ATy[j] = aty;
      }
    } else if (mode == 2) {
      // restart: u^{r+1,0} = ubar^{r,tau_r}
      x = V.xb[j];
      V.x[j] = x;
      V.x0[j] = x;
      if (HQ) {
        w = V.wb[j];
        qw = V.Qwb[j];
        V.w[j] = w;
        V.w0[j] = w;
        V.Qw[j] = qw;
        V.Qw0[j] = qw;
      }
      if (HA) {
        aty = V.ATyb[j];
        V.ATy[j] = aty;
        V.ATy0[j] = aty;
      }
    } else {
      x = V.x[j];
      if (HQ) {
        w = V.w[j];
        qw = V.Qw[j];
      }
      if (HA) aty = V.ATy[j];
    }
    // eq. (3.1)-(3.2)
    double g = -V.c[j];
    if (HQ) g -= qw;
    if (HA) g += aty;
    const double rz = fma(sigma, g, x);
    const double xbar = prox_phi(phi, rz, V.L[j], V.U[j], tau);
    V.xb[j] = xbar;
    if (ttest) V.zb[j] = (xbar - rz) * inv_sigma;
    // eq. (3.3)
    const double xh = fma(2.0, xbar, -x);
    V.xh[j] = xh;
    if (HQ) whout[j] = fma(c2, xh, c1 * w);
    else if (HA) V.v[j] = xh;
  }
}

template <int VAR>
__global__ void __launch_bounds__(kThreads) k_zx(Args a) {
  pdl_enter();
  zx_body<VAR>(a);
}

// ------------------------------------------------------------------------------------ factor pre-pass
// t = B_f x for every factor term (G lanes per row), t = F_g x for every dense term (one warp
// per row), x selected by `which` (PreSrc): wbar_{1/2} (and xbar on stopping tests), wbar, the
// restart difference A^*ybar - A^*y^{r,0}, the apply input, the power-method vector, or w_Q.
// TT: 0 one vector, 1 two (stopping test), 2 read C->ttest.
template <int G, int TT>
__device__ __forceinline__ void pre_body(const Args& a, int which) {
  const Ctrl* HPRQP_RESTRICT C = a.C;
  if (pre_in_step(which) && C->done) return;
  if (which == 2 && !C->restart_pending) return;
  if (which == 4 && C->pw_done) return;
  const QDev& Q = a.Q;
  const Vec& V = a.V;
  const bool two = (which == 0) && (TT == 1 || (TT == 2 && C->ttest));
  const double* x0 = which == PRE_WH ? (a.m > 0 ? V.wh : V.wb) : which == PRE_WB ? V.wb : which == PRE_AIN ? a.V.ain
                     : which == PRE_PV ? V.pv : which == PRE_W ? V.w : nullptr;
  const double* x1 = V.xb;
  double* t = pre_into_t1(which) ? V.t1 : V.t2;
  const int nt = Q.nfac + Q.ndense;
  const int64_t ffac = Q.nfac ? Q.toff[Q.nfac - 1] + Q.fac[Q.nfac - 1].rows : 0;  // rows of factor terms
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  // factor rows: G lanes per row
  {
    const int lane = threadIdx.x % G;
    const int64_t grp = gt / G, ngrp = gs / G;
    const int64_t ffac_pad = (ffac + ngrp - 1) / ngrp * ngrp;  // uniform trip count for the shuffles
    const L2Pol pol;
    for (int64_t r = grp; r < ffac_pad; r += ngrp) {
      double s0 = 0.0, s1 = 0.0;
      int term = 0;
      if (r < ffac)
        while (term + 1 < Q.nfac && r >= Q.toff[term + 1]) term++;
      // one-vector products of a tiled factor are formed by the tiled kernels; the products of
      // a thin factor for an inner step or the power method are formed inside the row pass
      // (q_csr_chunk)
      const bool step_src = which == PRE_WH || which == PRE_WB || which == PRE_W || which == PRE_PV;
      const bool mine = r < ffac && !(Q.tiled[term] && !two) && !(Q.inl[term] && step_src);
      if (mine) {
        const Csr& B = Q.fac[term];
        const int64_t rl = r - Q.toff[term];
        const int b = stream_i32(B.rp + rl, pol), e = stream_i32(B.rp + rl + 1, pol);
        // four entries' loads in flight before their (in-order) accumulation: the same sums
        // as one entry at a time, with four times the memory-level parallelism on long rows
        auto xval = [&](int c) {
          return which == 2 ? gather_f64(V.ATyb + c, pol) - gather_f64(V.ATy0 + c, pol) : gather_f64(x0 + c, pol);
        };
        int k = b + lane;
        for (; k + 3 * G < e; k += 4 * G) {
          const int c0 = stream_i32(B.ci + k, pol), c1 = stream_i32(B.ci + k + G, pol),
                    c2 = stream_i32(B.ci + k + 2 * G, pol), c3 = stream_i32(B.ci + k + 3 * G, pol);
          const double v0 = stream_f64(B.v + k, pol), v1 = stream_f64(B.v + k + G, pol),
                       v2 = stream_f64(B.v + k + 2 * G, pol), v3 = stream_f64(B.v + k + 3 * G, pol);
          const double a0 = xval(c0), a1 = xval(c1), a2 = xval(c2), a3 = xval(c3);
          s0 = fma(v0, a0, s0);
          s0 = fma(v1, a1, s0);
          s0 = fma(v2, a2, s0);
          s0 = fma(v3, a3, s0);
          if (two) {
            const double b0 = gather_f64(x1 + c0, pol), b1 = gather_f64(x1 + c1, pol),
                         b2 = gather_f64(x1 + c2, pol), b3 = gather_f64(x1 + c3, pol);
            s1 = fma(v0, b0, s1);
            s1 = fma(v1, b1, s1);
            s1 = fma(v2, b2, s1);
            s1 = fma(v3, b3, s1);
          }
        }
        if (k < e) {   // the remaining 0-3 entries, loads first, same order
          const bool h1 = k + G < e, h2 = k + 2 * G < e;
          const int c0 = stream_i32(B.ci + k, pol);
          const int c1 = h1 ? stream_i32(B.ci + k + G, pol) : c0;
          const int c2 = h2 ? stream_i32(B.ci + k + 2 * G, pol) : c0;
          const double v0 = stream_f64(B.v + k, pol);
          const double v1 = h1 ? stream_f64(B.v + k + G, pol) : 0.0;
          const double v2 = h2 ? stream_f64(B.v + k + 2 * G, pol) : 0.0;
          const double a0 = xval(c0);
          const double a1 = h1 ? xval(c1) : 0.0;
          const double a2 = h2 ? xval(c2) : 0.0;
          s0 = fma(v0, a0, s0);
          if (h1) s0 = fma(v1, a1, s0);
          if (h2) s0 = fma(v2, a2, s0);
          if (two) {
            const double b0 = gather_f64(x1 + c0, pol);
            const double b1 = h1 ? gather_f64(x1 + c1, pol) : 0.0;
            const double b2 = h2 ? gather_f64(x1 + c2, pol) : 0.0;
            s1 = fma(v0, b0, s1);
            if (h1) s1 = fma(v1, b1, s1);
            if (h2) s1 = fma(v2, b2, s1);
          }
        }
      }
      if (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
          s0 += __shfl_down_sync(0xffffffffu, s0, o, G);
          if (two) s1 += __shfl_down_sync(0xffffffffu, s1, o, G);
        }
      }
      if (lane == 0 && mine) {
        t[r] = s0;
        if (two) t[Q.tlen + r] = s1;
      }
    }
  }
  // dense rows: one warp per row
  if (Q.ndense) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = gt >> 5, nwarps = gs >> 5;
    for (int64_t r = ffac + warp; r < Q.tfd; r += nwarps) {
      int term = Q.nfac;
      while (term + 1 < nt && r >= Q.toff[term + 1]) term++;
      const int64_t rl = r - Q.toff[term];
      const double* F = Q.dense[term - Q.nfac] + (size_t)rl * Q.n;
      double s0 = 0.0, s1 = 0.0;
      for (int64_t j = lane; j < Q.n; j += 32) {
        const double xc = which == 2 ? V.ATyb[j] - V.ATy0[j] : x0[j];
        s0 = fma(F[j], xc, s0);
        if (two) s1 = fma(F[j], x1[j], s1);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        if (two) s1 += __shfl_down_sync(0xffffffffu, s1, o);
      }
      if (lane == 0) {
        t[r] = s0;
        if (two) t[Q.tlen + r] = s1;
      }
    }
  }
}

template <int G, int TT>
__global__ void __launch_bounds__(kThreads) k_pre(Args a, int which) {
  pdl_enter();
  pre_body<G, TT>(a, which);
}

// ------------------------------------------------------------------------------------ controller
// One pass of the Sec. 3.2 / Sec. 4.1 logic after an inner step; Ls: end-of-step sums,
// P3: y-step sums.  Runs on one thread.
__device__ __forceinline__ void controller(Ctrl& C, const double* Ls, const double* P3, CheckRec* hist = nullptr) {
  const long long kd = C.k + 1;
  bool bad = false;
  double R = 0.0;
  if (C.rtest) {
    // ||u - ubar||_M^2 = sigma th1 + th2/sigma + sigma^2 th3/(1+sigma lQ) + 2<dx, A^*dy - Q dw>
    const double th1 = C.lamA * P3[0] + C.lamQ * Ls[1] - 2.0 * Ls[2];
    const double R2 = C.sigma * th1 + Ls[0] * C.inv_sigma + C.sigma * Ls[3] + 2.0 * Ls[4];
    if (!isfinite(R2)) bad = true;
    R = sqrt(fmax(R2, 0.0));
    C.R = R;
  }
  if (C.ttest) {
    const double eta_p = P3[1] / (1.0 + fmax(C.b_inf, P3[2]));
    const double eta_d = Ls[5] / (1.0 + fmax(C.c_inf, fmax(Ls[6], Ls[7])));
    const double pobj = 0.5 * Ls[8] + Ls[9] + (C.phi != PHI_BOX ? C.lambda * Ls[10] : 0.0);
    const double dobj = -0.5 * Ls[8] + P3[3] - Ls[11];
    const double eta_g = fabs(pobj - dobj) / (1.0 + fmax(fabs(pobj), fabs(dobj)));
    C.eta_p = eta_p;
    C.eta_d = eta_d;
    C.eta_gap = eta_g;
    C.pobj = pobj;
    C.dobj = dobj;
    if (isnan(eta_p) || isnan(eta_d) || isnan(eta_g) || isinf(pobj) || isinf(dobj)) bad = true;
    const double rk = fmax(eta_p, fmax(eta_d, eta_g));
    if (hist) {
      CheckRec& h = hist[C.hist_n % kHistCap];
      h.iter = kd;
      h.restarts = C.r;
      h.sigma = C.sigma;
      h.eta_p = eta_p;
      h.eta_d = eta_d;
      h.eta_gap = eta_g;
      h.pobj = pobj;
      h.dobj = dobj;
      h.R = C.R;
      h.seconds = 1e-9 * (double)(global_ns() - C.t0_ns);
      C.hist_n++;
    }
    if (!bad && C.ladder_k[0] == 0 && rk <= 1e-4) {
      C.ladder_k[0] = kd;
      C.ladder_ns[0] = global_ns();
    }
    if (!bad && C.ladder_k[1] == 0 && rk <= 1e-6) {
      C.ladder_k[1] = kd;
      C.ladder_ns[1] = global_ns();
    }
    if (!bad && rk <= C.tol) {
      C.status = 0;
      C.done = 1;
      C.k = kd;
      return;
    }
    if (!bad && kd >= C.max_iter) {
      C.status = 1;
      C.done = 1;
      C.k = kd;
      return;
    }
  }
  if (bad) {
    C.status = 3;
    C.done = 1;
    C.k = kd;
    return;
  }
  bool restart = false;
  if (C.rtest && !C.restart_off) {
    if (C.t == 0) {
      C.R_r0 = R;
    } else {
      restart = (R <= C.alpha1 * C.R_r0) || (R <= C.alpha2 * C.R_r0 && R > C.R_prev) ||
                ((double)(C.t + 1) >= C.alpha3 * (double)kd);
    }
    C.R_prev = R;
  }
  if (restart) {
    if (C.r == 0) C.R_first = R;
    const double ratio = C.R_first > 0.0 ? R / C.R_first : 0.0;
    C.ratio = ratio;
    C.R_last = R;
    if (!C.sigma_fixed) C.restart_pending = 1;
    if (ratio <= C.ratio_tight) C.alpha3 = C.alpha3_tight;
    C.mode = 2;
    C.t = 0;
    C.r++;
  } else {
    halpern_weights(C, C.ha, C.hb);
    C.mode = 1;
    C.t++;
  }
  C.k = kd;
  C.rtest = !C.restart_off && ((C.t == 0) || ((C.k + 1) % C.restart_every == 0));
  C.ttest = ((C.k + 1) % C.check_every == 0) || (C.k + 1 >= C.max_iter);
  halpern_weights(C, C.fha, C.fhb);
}

__device__ __forceinline__ void set_handles(const Ctrl& C, const Handles& hd) {
  if (hd.has_rs) cudaGraphSetConditional(hd.rs_cur, (!C.done && C.restart_pending) ? 1u : 0u);
  if (hd.has_next) cudaGraphSetConditional(hd.sw_next, switch_value(C, hd));
}

// Per-row contributions to the R~ and stopping-rule sums (end of an inner step).
struct EndTerms {
  double s[kWL];
  __device__ void zero() {
#pragma unroll
    for (int i = 0; i < kWL; i++) s[i] = 0.0;
  }
};
constexpr unsigned kEndMax = (1u << 5) | (1u << 6) | (1u << 7);

__device__ __forceinline__ void end_row(EndTerms& T, const Args& a, int64_t j, bool rtest, bool ttest, bool HQ,
                                        bool HA, double Qwb_j) {
  const Vec& V = a.V;
  const double xb = V.xb[j];
  double atyb = 0.0;
  if (HA) atyb = V.ATyb[j];
  if (rtest) {
    const double dx = V.x[j] - xb;
    double qdw = 0.0, ady = 0.0;
    if (HQ) qdw = V.Qw[j] - Qwb_j;
    if (HA) ady = V.ATy[j] - atyb;
    T.s[0] = fma(dx, dx, T.s[0]);
    if (HQ) {
      const double dw = V.w[j] - V.wb[j];
      T.s[1] = fma(dw, qdw, T.s[1]);
      if (HA) {
        T.s[2] = fma(qdw, ady, T.s[2]);
        T.s[3] = fma(ady, V.Qwh[j] - Qwb_j, T.s[3]);
      }
    }
    T.s[4] = fma(dx, ady - qdw, T.s[4]);
  }
  if (ttest) {
    const double qxb = HQ ? V.Qxb[j] : 0.0;
    const double cj = V.c[j];
    // infinity norms in the original variables: every term of the dual residual is D^{-1}
    // times its scaled counterpart (x = D xs, y = E ys, z = D^{-1} zs)
    const double sc = V.isd ? V.isd[j] : 1.0;
    const double rd = iabs(atyb - qxb + V.zb[j] - cj) * sc;
    T.s[5] = imax(T.s[5], rd);
    T.s[6] = imax(T.s[6], iabs(atyb) * sc);
    T.s[7] = imax(T.s[7], iabs(qxb) * sc);
    T.s[8] = fma(xb, qxb, T.s[8]);
    T.s[9] = fma(cj, xb, T.s[9]);
    if (a.phi != PHI_BOX) T.s[10] += iabs(xb);
    T.s[11] += conj_phi_term(a.phi, V.zb[j], V.L[j], V.U[j], a.C->lambda);
  }
}

// Reduce the end terms of this block, elect the last block, run the controller.
template <bool ACTIVE>
__device__ __forceinline__ void end_iteration(EndTerms& T, const Args& a, const Handles& hd, bool active) {
  __shared__ double red[kWL * 32];
  if (ACTIVE && active) {
    block_reduce<kWL>(T.s, kEndMax, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < kWL; i++) a.partL[(size_t)blockIdx.x * kWL + i] = T.s[i];
    }
  }
  if (!last_block(&a.counters[0])) return;
  double Ls[kWL], P3[kW3];
#pragma unroll
  for (int i = 0; i < kWL; i++) Ls[i] = 0.0;
#pragma unroll
  for (int i = 0; i < kW3; i++) P3[i] = 0.0;
  if (ACTIVE && active) {
    reduce_partials<kWL>(a.partL, gridDim.x, kWL, kEndMax, Ls, red);
    __syncthreads();
    if (a.m > 0) reduce_partials<kW3>(a.part3, a.nbM, kW3, 0x6u, P3, red);
  }
  if (threadIdx.x == 0) {
    controller(*a.C, Ls, P3, a.hist);
    set_handles(*a.C, hd);
  }
}

// ------------------------------------------------------------------------------------ row kernels
template <int G, int KIND, int VAR>
__device__ __forceinline__ void rows_body(const Args& a, const Handles& hd) {
  Ctrl* HPRQP_RESTRICT C = a.C;
  if (step_kind(KIND) && C->done) return;
  if ((KIND == K_POWER_Q || KIND == K_POWER_A || KIND == K_APPLY_AT_P) && C->pw_done) return;
  __shared__ double rs0[kChunk];
  __shared__ double rs1[kChunk];
  const Vec& V = a.V;
  const QDev& Q = a.Q;
  const bool HQ = Q.present(), HA = a.m > 0;
  // the fused passes belong to a plain step; their VAR is the variant of the next step
  constexpr bool FUSED = (KIND == K_ATH || KIND == K_Q2H);
  const bool ttest = (KIND <= K_Q2) ? var_ttest<VAR>(C) : false;
  const bool rtest = (KIND <= K_Q2) ? var_rtest<VAR>(C) : false;
  constexpr bool RED = (VAR != VAR_PLAIN) && !FUSED;   // the variant carries reduction code
  const int64_t rows = (KIND == K_A1 || KIND == K_APPLY_A || KIND == K_POWER_A) ? a.m : a.n;
  const int64_t nchunks = (rows + kChunk - 1) / kChunk;
  const double sigma = C->sigma, s = C->s, slA = C->slA, inv_slA = C->inv_slA;
  const int mode = C->mode;
  // the fused passes apply the Halpern step that follows this one (the weights the controller
  // will set at the end of this step, computed by it with this step's t and k)
  const double ha = FUSED ? C->fha : C->ha, hb = FUSED ? C->fhb : C->hb;
  const bool last_of_iter = (KIND == K_Q2) || (KIND == K_Q2H) || (KIND == K_Q1 && !HA) || (KIND == K_AT && !HQ);
  EndTerms T;
  T.zero();
  double y3[kW3] = {0.0, 0.0, 0.0, 0.0};
  double pw[kWP] = {0.0, 0.0};

  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t row0 = ch * kChunk;
    // ---- phase 1: CSR row sums into shared memory
    if (KIND == K_Q1) {
      const double* src = HA ? V.wh : V.wb;
      if (RED && ttest) q_csr_chunk<G, 2>(Q, row0, src, V.xb, V.t1, V.t1 + Q.tlen, rs0, rs1, true);
      else q_csr_chunk<G, 1>(Q, row0, src, nullptr, V.t1, nullptr, rs0, rs1, true);
    } else if (KIND == K_Q2) {
      q_csr_chunk<G, 1>(Q, row0, V.wb, nullptr, V.t2, nullptr, rs0, rs1, true);
    } else if (KIND == K_Q2H) {
      q_csr_chunk<G, 1>(Q, row0, V.w, nullptr, V.t2, nullptr, rs0, rs1, true);
    } else if (KIND == K_APPLY_Q) {
      q_csr_chunk<G, 1>(Q, row0, V.ain, nullptr, V.t1, nullptr, rs0, rs1);
    } else if (KIND == K_POWER_Q) {
      q_csr_chunk<G, 1>(Q, row0, V.pv, nullptr, V.t1, nullptr, rs0, rs1, true);
    } else if (KIND == K_A1) {
      if (RED && ttest) csr_chunk<G, 2>(a.A, row0, V.v, V.xb, rs0, rs1, false);
      else csr_chunk<G, 1>(a.A, row0, V.v, nullptr, rs0, rs1, false);
    } else if (KIND == K_APPLY_A) {
      csr_chunk<G, 1>(a.A, row0, V.ain, nullptr, rs0, rs1, false);
    } else if (KIND == K_POWER_A) {
      csr_chunk<G, 1>(a.A, row0, V.ptmp, nullptr, rs0, rs1, false);
    } else if (KIND == K_AT || KIND == K_ATH) {
      csr_chunk<G, 1>(a.AT, row0, V.yb, nullptr, rs0, rs1, false);
    } else if (KIND == K_APPLY_AT) {
      csr_chunk<G, 1>(a.AT, row0, V.ain, nullptr, rs0, rs1, false);
    } else if (KIND == K_APPLY_AT_P) {
      csr_chunk<G, 1>(a.AT, row0, V.pv, nullptr, rs0, rs1, false);
    }
    // With one lane per row (G = 1) every part of phase 1 leaves row r's sum to thread r, the
    // thread that reads it in phase 2 and overwrites it in the next chunk: no barrier is needed,
    // and a warp whose rows are short does not wait for the block's slowest row.  The staged and
    // SELL forms (G = 0, -1) and groups of G > 1 lanes write sums of other threads' rows.
    if constexpr (G != 1) __syncthreads();
    // ---- phase 2: thread per row, full warps
    const int64_t j = row0 + threadIdx.x;
    if (j < rows) {
      const double r0 = rs0[threadIdx.x];
      if (KIND == K_Q1) {
        const double* src = HA ? V.wh : V.wb;
        const double qwh = r0 + q_local(Q, j, src, V.t1, true, !(RED && ttest));
        if (RED && ttest) V.Qxb[j] = rs1[threadIdx.x] + q_local(Q, j, V.xb, V.t1 + Q.tlen, true, false);
        if (HA) {
          // v = what + sigma (Q w - Q wbar_{1/2})   (eq. (3.5), second form)
          V.v[j] = fma(sigma, V.Qw[j] - qwh, V.xh[j]);
          if (RED && rtest) V.Qwh[j] = qwh;
        } else {
          V.Qwb[j] = qwh;  // m = 0: wbar = wbar_{1/2}
          if (RED) end_row(T, a, j, rtest, ttest, HQ, HA, qwh);
        }
      } else if (KIND == K_Q2) {
        const double qwb = r0 + q_local(Q, j, V.wb, V.t2, true, true);
        V.Qwb[j] = qwb;
        if (RED) end_row(T, a, j, rtest, ttest, HQ, HA, qwb);
      } else if (KIND == K_Q2H) {
        // Q w of the new iterate (K_ATH wrote w), then the next step's elementwise pass: the
        // Halpern step on x with 2 xbar - x = what, eqs. (3.1)-(3.3) as in k_zx
        const double qw = r0 + q_local(Q, j, V.w, V.t2, true, true);
        V.Qw[j] = qw;
        const double x = fma(hb, V.xh[j], ha * V.x0[j]);
        double g = -V.c[j];
        g -= qw;
        g += V.ATy[j];
        const double rz = fma(sigma, g, x);
        const double xbar = prox_phi(a.phi, rz, V.L[j], V.U[j], C->tau);
        const double xh = fma(2.0, xbar, -x);
        V.xh[j] = xh;
        V.wh[j] = fma(C->c2, xh, C->c1 * V.w[j]);
        if (VAR != VAR_PLAIN) {   // the next step evaluates R~ or the stopping rule
          V.xb[j] = xbar;
          V.x[j] = x;
        }
        if (VAR == VAR_T) V.zb[j] = (xbar - rz) * C->inv_sigma;
      } else if (KIND == K_A1) {
        // Halpern / restart on y, then eq. (3.5)
        double y;
        if (mode == 1) {
          y = fma(hb, fma(2.0, V.yb[j], -V.y[j]), ha * V.y0[j]);
          V.y[j] = y;
        } else if (mode == 2) {
          y = V.yb[j];
          V.y[j] = y;
          V.y0[j] = y;
        } else {
          y = V.y[j];
        }
        const double lo = V.l[j], hi = V.u[j];
        const double ry = fma(-slA, y, r0);
        const double yb = (iclamp(ry, lo, hi) - ry) * inv_slA;
        V.yb[j] = yb;
        if (RED && rtest) {
          const double dy = y - yb;
          y3[0] = fma(dy, dy, y3[0]);
        }
        if (RED && ttest) {
          const double ax = rs1[threadIdx.x];
          const double sc = V.ise ? V.ise[j] : 1.0;   // A x = E^{-1} (A_s xs)
          y3[1] = imax(y3[1], iabs(ax - iclamp(ax, lo, hi)) * sc);
          y3[2] = imax(y3[2], iabs(ax) * sc);
          double t = 0.0;
          if (igt0(yb)) t = lo * yb;
          else if (ilt0(yb)) t = hi * yb;
          y3[3] += t;
        }
      } else if (KIND == K_AT) {
        V.ATyb[j] = r0;
        if (HQ) {
          // wbar = wbar_{1/2} + sigma/(1+sigma lQ) (A^* ybar - A^* y)   (eq. (3.3))
          V.wb[j] = fma(s, r0 - V.ATy[j], V.wh[j]);
        } else if (RED) {
          end_row(T, a, j, rtest, ttest, HQ, HA, 0.0);
        }
      } else if (KIND == K_ATH) {
        // wbar as in K_AT, then the Halpern step of the next iteration on w_Q and A^* y,
        // u = 1/(i+2) u^{r,0} + (i+1)/(i+2) (2 ubar - u); wbar and A^* ybar stay in registers
        const double aty = V.ATy[j];
        const double wb = fma(s, r0 - aty, V.wh[j]);
        V.ATy[j] = fma(hb, fma(2.0, r0, -aty), ha * V.ATy0[j]);
        V.w[j] = fma(hb, fma(2.0, wb, -V.w[j]), ha * V.w0[j]);
      } else if (KIND == K_APPLY_Q) {
        V.aout[j] = r0 + q_local(Q, j, V.ain, V.t1, true, true);
      } else if (KIND == K_APPLY_A || KIND == K_APPLY_AT) {
        V.aout[j] = r0;
      } else if (KIND == K_APPLY_AT_P) {
        V.ptmp[j] = r0;
      } else if (KIND == K_POWER_Q || KIND == K_POWER_A) {
        // the source is the previous product w, unnormalised: v = w / ||w|| = pw_scale w, and
        // the operator is linear, so Q v = pw_scale (Q w) (A A^* likewise)
        const double sc = C->pw_scale;
        const double wv = sc * (KIND == K_POWER_Q ? r0 + q_local(Q, j, V.pv, V.t1, true, true) : r0);
        V.pw[j] = wv;
        pw[0] = fma(sc * V.pv[j], wv, pw[0]);
        pw[1] = fma(wv, wv, pw[1]);
      }
    }
    if constexpr (G != 1) __syncthreads();   // rs0 / rs1 are reused by the next chunk
  }

  // ---- block reductions / controllers
  if (KIND == K_A1 && RED) {
    __shared__ double red3[kW3 * 32];
    if (rtest || ttest) {
      block_reduce<kW3>(y3, 0x6u, red3);
      if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < kW3; i++) a.part3[(size_t)blockIdx.x * kW3 + i] = y3[i];
      }
    }
  }
  if (last_of_iter) end_iteration<RED>(T, a, hd, rtest || ttest);
  if (KIND == K_POWER_Q || KIND == K_POWER_A) {
    __shared__ double redp[kWP * 32];
    block_reduce<kWP>(pw, 0u, redp);
    if (threadIdx.x == 0) {
      a.partP[(size_t)blockIdx.x * kWP] = pw[0];
      a.partP[(size_t)blockIdx.x * kWP + 1] = pw[1];
    }
    if (last_block(&a.counters[2])) {
      double tot[kWP];
      reduce_partials<kWP>(a.partP, gridDim.x, kWP, 0u, tot, redp);
      if (threadIdx.x == 0) {
        // Rayleigh quotient of the unit vector v, Sec. 4.1 power method
        const double lnew = tot[0], nw = sqrt(tot[1]);
        if (nw == 0.0 || !isfinite(nw)) {
          C->pw_lam = 0.0;
          C->pw_done = 1;
          C->pw_scale = 0.0;
        } else {
          const bool conv = (C->pw_it > 0) && fabs(lnew - C->pw_lam) <= C->pw_tol * fabs(lnew);
          C->pw_lam = lnew;
          C->pw_scale = 1.0 / nw;
          C->pw_it++;
          if (conv || C->pw_it >= C->pw_max) C->pw_done = 1;
        }
      }
    }
  }
}

template <int G, int KIND, int VAR>
// plain steps keep six blocks per SM resident (at most 40 registers): their passes are
// latency-bound gathers, so occupancy matters more than a few extra registers; the variants that
// reduce (R~ and stopping tests) keep four (at most 64 registers: unbounded they took 80-112
// registers and ran at a quarter of the SM's warps, twice as long as the plain passes)
__global__ void __launch_bounds__(kThreads, (VAR == VAR_PLAIN || KIND == K_ATH || KIND == K_Q2H) ? 6 : 4)
    k_rows(Args a, Handles hd) {
  pdl_enter();
  rows_body<G, KIND, VAR>(a, hd);
}

// ------------------------------------------------------------------------------------ restart (Alg. 5)
__device__ __forceinline__ void sigma_argmin_dev(double t1, double t2, double t3, double lq, int golden,
                                                 double* out) {
  double hi = sqrt(t2 / t1);
  if (t3 <= 0.0 || lq <= 0.0) {
    *out = hi;
    return;
  }
  double lo = sqrt(t2 / (t1 + t3 / lq));
  if (!golden) {
    for (int it = 0; it < 200 && (hi - lo) > 4.0e-16 * hi; it++) {
      const double mid = 0.5 * (lo + hi);
      const double d = 1.0 + lq * mid;
      const double fp = t1 - t2 / (mid * mid) + t3 * mid * (2.0 + lq * mid) / (d * d);
      if (fp > 0.0) hi = mid;
      else lo = mid;
    }
    *out = 0.5 * (lo + hi);
    return;
  }
  const double gr = 0.6180339887498949;
  double A = log(lo), B = log(hi);
  double x1 = B - gr * (B - A), x2 = A + gr * (B - A);
  auto f = [&](double u) {
    const double sv = exp(u);
    return t1 * sv + t2 / sv + sv * sv * t3 / (1.0 + lq * sv);
  };
  double f1 = f(x1), f2 = f(x2);
  for (int it = 0; it < 200 && (B - A) > 1e-12; it++) {
    if (f1 < f2) {
      B = x2; x2 = x1; f2 = f1;
      x1 = B - gr * (B - A);
      f1 = f(x1);
    } else {
      A = x1; x1 = x2; f1 = f2;
      x2 = A + gr * (B - A);
      f2 = f(x2);
    }
  }
  *out = exp(0.5 * (A + B));
}

template <int G>
__device__ __forceinline__ void restart_body(const Args& a) {
  Ctrl* HPRQP_RESTRICT C = a.C;
  if (C->done || !C->restart_pending) return;
  __shared__ double rs0[kChunk];
  __shared__ double red[kWR * 32];
  const Vec& V = a.V;
  const QDev& Q = a.Q;
  const bool HQ = Q.present(), HA = a.m > 0;
  double S[kWR] = {0.0, 0.0, 0.0, 0.0, 0.0};
  const int64_t nchunks = (a.n + kChunk - 1) / kChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t row0 = ch * kChunk;
    // d = A^*ybar - A^*y^{r,0}; explicit CSR part of <d, Q d> (gathered on the fly)
    if (HQ && HA && Q.csr.rows) {
      const int lane = threadIdx.x % G, grp = threadIdx.x / G;
      for (int rr = grp; rr < kChunk; rr += kThreads / G) {
        const int64_t row = row0 + rr;
        double s0 = 0.0;
        if (row < a.n) {
          for (int k = Q.csr.rp[row] + lane; k < Q.csr.rp[row + 1]; k += G) {
            const int c = Q.csr.ci[k];
            s0 = fma(Q.csr.v[k], V.ATyb[c] - V.ATy0[c], s0);
          }
        }
        for (int o = G / 2; o > 0; o >>= 1) s0 += __shfl_down_sync(0xffffffffu, s0, o, G);
        if (lane == 0 && row < a.n) rs0[rr] = s0;
      }
    } else {
      rs0[threadIdx.x] = 0.0;
    }
    __syncthreads();
    const int64_t j = row0 + threadIdx.x;
    if (j < a.n) {
      const double dx = V.xb[j] - V.x0[j];
      S[3] = fma(dx, dx, S[3]);
      if (HQ) {
        const double dw = V.wb[j] - V.w0[j];
        const double qdw = V.Qwb[j] - V.Qw0[j];
        S[1] = fma(dw, qdw, S[1]);
        if (HA) {
          const double d = V.ATyb[j] - V.ATy0[j];
          S[2] = fma(qdw, d, S[2]);
          // <d, (diag + band + CSR) d>; the factor parts come from ||t2||^2 below
          double qd = rs0[threadIdx.x];
          if (Q.diag) qd = fma(Q.diag[j], d, qd);
          for (int k = 0; k < Q.ndia; k++) {
            const int o = Q.dia_off[k];
            const double* dg = Q.dia + (size_t)k * Q.n;
            if (o == 0) {
              qd = fma(dg[j], d, qd);
            } else {
              if (j + o < a.n) qd = fma(dg[j], V.ATyb[j + o] - V.ATy0[j + o], qd);
              if (j - o >= 0) qd = fma(dg[j - o], V.ATyb[j - o] - V.ATy0[j - o], qd);
            }
          }
          if (Q.qap_d) qd += V.t2[Q.qap_off + j];   // (Q_qap d)_j from the pre-pass
          S[4] = fma(d, qd, S[4]);
        }
      }
    }
    __syncthreads();
  }
  // ||B_f d||^2 and ||F_g d||^2 from the pre-pass, and ||ybar - y^{r,0}||^2
  const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  if (HQ && HA) {
    for (int64_t r = gt; r < Q.tfd; r += gs) S[4] = fma(V.t2[r], V.t2[r], S[4]);
  }
  for (int64_t i = gt; i < a.m; i += gs) {
    const double dy = V.yb[i] - V.y0[i];
    S[0] = fma(dy, dy, S[0]);
  }
  block_reduce<kWR>(S, 0u, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < kWR; i++) a.partR[(size_t)blockIdx.x * kWR + i] = S[i];
  }
  if (!last_block(&a.counters[1])) return;
  double tot[kWR];
  reduce_partials<kWR>(a.partR, gridDim.x, kWR, 0u, tot, red);
  if (threadIdx.x == 0) {
    // Algorithm 5: theta~ of eq. (3.11), floors, argmin of eq. (3.12), smoothing
    double th1 = C->lamA * tot[0] + C->lamQ * tot[1] - 2.0 * tot[2];
    double th2 = tot[3];
    const double th3 = tot[4];
    th1 = fmax(th1, 1e-12);
    th2 = fmax(th2, 1e-12);
    double snew;
    sigma_argmin_dev(th1, th2, th3, C->lamQ, C->sigma_golden, &snew);
    const double beta = exp(-C->ratio);
    const double sig = exp(beta * log(snew) + (1.0 - beta) * log(C->sigma));
    if (!isfinite(sig) || !(sig > 0.0)) {
      C->status = 3;
      C->done = 1;
    } else {
      set_sigma(*C, sig);
    }
    C->restart_pending = 0;
  }
}

template <int G>
__global__ void __launch_bounds__(kThreads) k_restart(Args a) {
  pdl_enter();
  restart_body<G>(a);
}

using RowKernel = void (*)(Args, Handles);

// per-translation-unit kernel tables (rows_q.cu, rows_a.cu, rows_at.cu)
RowKernel row_kernel_q(int kind, int var, int G);
RowKernel row_kernel_a(int kind, int var, int G);
RowKernel row_kernel_at(int kind, int var, int G);

// kinds whose CSR pass is one matrix with a SELL copy (A or A^T)
constexpr bool sell_kind(int kind) {
  return kind == K_A1 || kind == K_APPLY_A || kind == K_POWER_A || kind == K_AT || kind == K_APPLY_AT ||
         kind == K_APPLY_AT_P || kind == K_ATH;
}

template <int KIND>
RowKernel pick_row(int var, int G) {
#define HPRQP_ROW_G(VAR)                                        \
  switch (G) {                                                  \
    case -1:                                                    \
      if constexpr (sell_kind(KIND)) return k_rows<-1, KIND, VAR>; \
      else return nullptr;                                      \
    case 0: return k_rows<0, KIND, VAR>;                        \
    case 1: return k_rows<1, KIND, VAR>;                        \
    case 2: return k_rows<2, KIND, VAR>;                        \
    case 4: return k_rows<4, KIND, VAR>;                        \
    case 8: return k_rows<8, KIND, VAR>;                        \
    case 16: return k_rows<16, KIND, VAR>;                      \
    default: return k_rows<32, KIND, VAR>;                      \
  }
  if constexpr (KIND == K_ATH) {
    HPRQP_ROW_G(VAR_PLAIN)
  } else if constexpr (KIND == K_Q2H) {
    switch (var) {
      case VAR_PLAIN: { HPRQP_ROW_G(VAR_PLAIN) }
      case VAR_R: { HPRQP_ROW_G(VAR_R) }
      default: { HPRQP_ROW_G(VAR_T) }
    }
  } else if constexpr (KIND > K_Q2) {
    HPRQP_ROW_G(VAR_PLAIN)
  } else {
    switch (var) {
      case VAR_PLAIN: { HPRQP_ROW_G(VAR_PLAIN) }
      case VAR_R: { HPRQP_ROW_G(VAR_R) }
      case VAR_T: { HPRQP_ROW_G(VAR_T) }
      default: { HPRQP_ROW_G(VAR_RUNTIME) }
    }
  }
#undef HPRQP_ROW_G
}

}  // namespace hprqp
