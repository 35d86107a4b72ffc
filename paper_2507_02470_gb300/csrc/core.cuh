// Device-side data structures and small helpers of the HPR-QP library (sm_103a, FP64).
//
// On GB300 the FP64 pipe retires one warp instruction per ~19 SM cycles whatever the
// number of active lanes, so the kernels keep every FP64 instruction on full warps and do
// comparisons, clamps and max-reductions on the integer pipe (bit-exact with the FP64
// operations for non-NaN inputs).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hprqp {

constexpr int kMaxDia = 8;
constexpr int kMaxFac = 4;
constexpr int kMaxDense = 4;
constexpr int kChunk = 256;      // rows per block pass of the row kernels (= block size)
constexpr int kThreads = 256;

enum Phi { PHI_BOX = 0, PHI_L1 = 1, PHI_L1_BOX = 2 };

struct Csr {
  int64_t rows = 0, cols = 0, nnz = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const double* v = nullptr;
  // optional SELL-32 copy (A and A^T): rows sorted by length inside each 256-row chunk, slices
  // of 32 rows, entry m of a slice's lane l at soff[slice] + 32 m + l, zero-padded
  const int* soff = nullptr;    // slices + 1
  const int* sperm = nullptr;   // slices * 32: row of each lane, -1 for padding
  const int* sci = nullptr;
  const double* sv = nullptr;
};

// Shared-memory-tiled copy of a factor term B_f (p x n) for products with one vector: t = B x
// runs per column tile of x (kTileW entries held in shared memory) into per-tile partial sums,
// u = B^T t per tile of t; both gather from shared memory instead of L2.  Each tile of a
// matrix M (B or B^T) is stored as sliced ELLPACK with sorting (SELL-32-512): rows taken in
// windows of 512, sorted inside the window by their entry count in the tile, cut into slices
// of 32 rows (one per lane of a warp), entry m of a slice's lane l at off + 32 m + l, padded
// with zero values to the longest row of the slice.  Column indices are tile-local (16 bits).
constexpr int kTileW = 25600;   // doubles per shared-memory tile (200 KB)
constexpr int kSellC = 32;      // rows per slice
constexpr int kSellWin = 512;   // rows per sorting window (16 slices)
struct SellTiles {
  int64_t rows = 0;               // rows of M
  int ntile = 0;                  // column tiles of M
  int64_t nsl = 0;                // slices per tile: ceil(rows / 32)
  const int* off = nullptr;       // ntile x (nsl + 1) entry offsets of the slices
  const int* perm = nullptr;      // ntile x (nsl * 32): row of each slice lane, -1 for padding
  const unsigned short* col = nullptr;   // tile-local columns
  const double* val = nullptr;
};
struct TiledFac {
  int64_t p = 0;
  int nrange = 0;                 // blocks per column tile of B (windows split among them)
  SellTiles b;                    // B (p x n): tiles over the columns of B (entries of x)
  SellTiles bt;                   // B^T (n x p): tiles over the rows of B (entries of t)
  double* part = nullptr;         // b.ntile x p partial sums of B x, one row per column tile
};

// Q = diag(d) + sym band + CSR + sum_f B_f^T B_f + sum_g F_g^T F_g   (Sec. 1: Q may be
// matrix-free).  The factor intermediates t = B v, F v live in one buffer at toff[].
struct QDev {
  int64_t n = 0;
  const double* diag = nullptr;
  Csr csr;                               // rows == 0: absent
  int ndia = 0;
  int dia_off[kMaxDia] = {0};
  const double* dia = nullptr;           // ndia x n, dia[k*n+i] = Q[i][i+off_k]
  int nfac = 0;
  Csr fac[kMaxFac];                      // B_f (p x n)
  Csr fact[kMaxFac];                     // B_f^T (n x p)
  int ndense = 0;
  int64_t dense_p[kMaxDense] = {0};
  const double* dense[kMaxDense] = {nullptr};   // F_g row-major p x n
  int64_t toff[kMaxFac + kMaxDense] = {0};
  // QAP term (Sec. 4.5): Ahat, Bhat, S, T (d x d each, contiguous); its product Q_qap x is
  // formed before a pass (the FP64 contractions of qap.cu) into the intermediate buffer at
  // qap_off, like B_f x
  int64_t qap_d = 0;
  const double* qap = nullptr;
  double* qap_tmp = nullptr;    // d x d scratch (Ahat X)
  double* qap_in = nullptr;     // n scratch (restart difference)
  double* qap_part = nullptr;   // qap_splits x d x d partial tiles of a split contraction
  unsigned* qap_count = nullptr;   // one counter per 32 x 32 tile of the result
  int qap_splits = 1;           // blocks sharing the K range of one tile
  int64_t qap_off = 0;
  // factor terms with a tiled copy: their one-vector products (t = B x, then u = B^T t into
  // the intermediate buffer at uoff) run in the tiled kernels; the two-vector products of a
  // stopping test keep the CSR pre-pass and row pass
  int tiled[kMaxFac] = {0};
  // thin factor terms (few rows of B meet any row of B^T: sum over B's rows of their squared
  // lengths is small against n): the inner step's products form (B x)_r from row r of B inside
  // the row pass that needs it, with no pre-pass; other products (apply, power method, restart
  // difference) still use the pre-pass
  int inl[kMaxFac] = {0};
  TiledFac tf[kMaxFac];
  int64_t uoff[kMaxFac] = {0};
  int64_t tfd = 0;              // intermediate rows of the factor and dense terms
  int64_t tlen = 0;             // tfd, plus n for the QAP product
  __host__ __device__ bool present() const { return diag || csr.rows || ndia || nfac || ndense || qap_d; }
  __host__ __device__ bool has_pre() const { return nfac || ndense || qap_d; }   // products before a pass
  __host__ __device__ bool has_fd() const { return nfac || ndense; }             // ... by k_pre
};

// One stopping test of a solve (the controller appends it to a ring of kHistCap records).
constexpr int kHistCap = 512;
struct CheckRec {
  long long iter, restarts;
  double sigma, eta_p, eta_d, eta_gap, pobj, dobj, R, seconds;
};

// Scalars of the running iteration.  Written by the controller (the last block of the
// last kernel of an iteration) and by the restart kernel; read by every kernel.
struct Ctrl {
  // per-iteration scalars
  double sigma, inv_sigma;
  double c1, c2, s;          // sigma lQ/(1+sigma lQ), 1/(1+sigma lQ), sigma/(1+sigma lQ)
  double slA, inv_slA;       // sigma lA and its reciprocal
  double tau;                // sigma * lambda (l1 threshold)
  double ha, hb;             // pending Halpern weights 1/(i+2), (i+1)/(i+2)
  double fha, fhb;           // weights of the Halpern step after this one (if no restart), for
                             // the fused passes: set with t and k, so no kernel thread divides
  int mode;                  // update at the start of this iteration: 0 none, 1 Halpern, 2 restart
  int rtest, ttest;          // this iteration evaluates R~ / the stopping rule
  int done;                  // kernels return at entry
  int restart_pending;       // the sigma update must run before the next iteration
  int status;
  long long k, t, r;
  // restart bookkeeping (Sec. 3.2)
  double R_r0, R_prev, R_first, R_last, alpha3, ratio;
  // constants
  double lamA, lamQ, lambda, tol;
  double alpha1, alpha2, alpha3_tight, ratio_tight;
  double c_inf, b_inf;
  long long max_iter, check_every, restart_every;
  int halpern_total, restart_off, sigma_fixed, sigma_golden;
  int has_A, has_Q, phi;
  // results of the last stopping test
  double eta_p, eta_d, eta_gap, pobj, dobj, R;
  // tolerance ladder (Sec. 4 reports 1e-4, 1e-6, 1e-8): first stopping test meeting 1e-4 / 1e-6,
  // with the device time stamp (%globaltimer, ns) of that test and of the first step
  long long ladder_k[2];
  unsigned long long ladder_ns[2], t0_ns;
  long long hist_n;            // stopping tests recorded so far (ring of kHistCap)
  // power method state
  double pw_lam, pw_scale;
  long long pw_it, pw_max;
  double pw_tol;
  int pw_done;
};

// ---------------------------------------------------------------------------- int-pipe FP64 helpers
// Monotone map of a double (non-NaN) onto a signed 64-bit key: a < b  <=>  key(a) < key(b)
__device__ __forceinline__ long long dkey(double a) {
  long long b = __double_as_longlong(a);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ double imax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }
__device__ __forceinline__ double imin(double a, double b) { return dkey(a) <= dkey(b) ? a : b; }
__device__ __forceinline__ double iclamp(double v, double lo, double hi) { return imin(imax(v, lo), hi); }
__device__ __forceinline__ double iabs(double a) {
  return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ bool igt0(double a) { return __double_as_longlong(a) > 0; }        // a > +0
__device__ __forceinline__ bool ilt0(double a) {                                             // a < -0
  return __double_as_longlong(a) < 0 && (__double_as_longlong(a) & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool iisinf(double a) {
  return (__double_as_longlong(a) & 0x7fffffffffffffffLL) == 0x7ff0000000000000LL;
}

// ---------------------------------------------------------------------------- block reductions
// Deterministic: fixed lane/warp order.  op 0 = sum, 1 = max of non-negative values.
template <int NT>
__device__ __forceinline__ void block_reduce(double (&v)[NT], const unsigned maxmask, double* smem) {
  // smem: at least NT * 32 doubles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NT; i++) {
    double a = v[i];
    bool mx = (maxmask >> i) & 1u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double b = __shfl_down_sync(0xffffffffu, a, o);
      a = mx ? imax(a, b) : a + b;
    }
    if (lane == 0) smem[i * 32 + warp] = a;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int i = 0; i < NT; i++) {
      bool mx = (maxmask >> i) & 1u;
      double a = lane < nw ? smem[i * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double b = __shfl_down_sync(0xffffffffu, a, o);
        a = mx ? imax(a, b) : a + b;
      }
      if (lane == 0) v[i] = a;
    }
  }
  __syncthreads();
}

// Last-block election: every block stores its partials, then the last one to arrive
// returns true (and has visibility of all partials).
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(counter, 1u);
    am_last = (prev == gridDim.x - 1);
    if (am_last) *counter = 0;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Sum (or max) of `nblocks` partial rows of width W, term i at part[b*W + i]; every thread of
// the block takes part; the result is valid in out[] of thread 0.  Fixed order.
template <int NT>
__device__ __forceinline__ void reduce_partials(const double* part, int nblocks, int W, unsigned maxmask,
                                                double (&out)[NT], double* smem) {
#pragma unroll
  for (int i = 0; i < NT; i++) out[i] = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int i = 0; i < NT; i++) {
      double p = __ldcg(part + (size_t)b * W + i);
      out[i] = ((maxmask >> i) & 1u) ? imax(out[i], p) : out[i] + p;
    }
  }
  block_reduce<NT>(out, maxmask, smem);
}

}  // namespace hprqp
