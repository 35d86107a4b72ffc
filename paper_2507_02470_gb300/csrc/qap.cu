// The QAP-relaxation operator of Sec. 4.5 as two FP64 contractions:
//
//   Q vec(X) = vec(Ahat X Bhat - S X - X T),   X = reshape(x, d, d) column-major,
//
//   stage 1:  T1  = Ahat X
//   stage 2:  out = T1 Bhat - S X - X T = [T1 | S | X] [Bhat ; -X ; -T]
//
// so stage 2 is one contraction over K = 3d whose three operand pairs are summed in registers
// (the -SX - XT terms fused into the second product).  All matrices are d x d column-major
// (Ahat, Bhat, S, T are symmetric, so either storage order reads the same).
//
// On GB300 FP64 issues one warp instruction per 19 SM cycles, so an FP64 contraction is bound
// by FMA issue, not by memory or shared-memory bandwidth: each block computes a 32 x 32 tile of
// the result with 64 threads, 4 x 4 accumulators per thread (16 independent FMAs per k), the
// operands staged through shared memory 16 k at a time with the next stage's loads held in
// registers during the current stage's FMAs.  Small d give few tiles, so the K range is split
// across blocks; each split writes its partial tile and the last split to finish (a counter
// per tile) sums the partials in split order, so results do not depend on timing.
#include <cuda_runtime.h>

#include <algorithm>

#include "solver.cuh"

namespace hprqp {

namespace {

constexpr int kQT = 32;        // tile edge
constexpr int kQK = 16;        // k per shared-memory stage
constexpr int kQThreads = 64;  // 8 x 8 threads, 4 x 4 outputs each

// One operand pair of a contraction: C += sign * A B (A, B column-major d x d).
struct Pair {
  const double* A;
  const double* B;
  double sign;
};

struct Gemm {
  Pair p[3];
  int npair;
  int d;
  double* C;          // d x d result
  double* part;       // splits x d x d partial tiles (when splits > 1)
  unsigned* count;    // one counter per tile (when splits > 1), zero between launches
  int splits;
};

__global__ void __launch_bounds__(kQThreads) k_qap_gemm(Gemm g) {
  __shared__ double As[kQK][kQT];   // As[k][i] = A[i0 + i, k0 + k]
  __shared__ double Bs[kQK][kQT];   // Bs[k][j] = B[k0 + k, j0 + j]
  __shared__ bool last;
  const int d = g.d;
  const int tiles_i = (d + kQT - 1) / kQT;
  const int tile = blockIdx.x % (tiles_i * tiles_i), split = blockIdx.x / (tiles_i * tiles_i);
  const int i0 = (tile % tiles_i) * kQT, j0 = (tile / tiles_i) * kQT;
  const int t = threadIdx.x, tr = t % 8, tc = t / 8;
  // this split's share of the K range [0, npair * d), in whole stages of kQK
  const int kstages = g.npair * ((d + kQK - 1) / kQK);
  const int s0 = (int)((long long)split * kstages / g.splits), s1 = (int)((long long)(split + 1) * kstages / g.splits);
  const int per_pair = (d + kQK - 1) / kQK;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
  // loads of one stage: 512 entries of A's tile and 512 of B's, 8 each per thread; entry e of
  // the A tile is (i = e % 32, k = e / 32), of the B tile (k = e % 16, j = e / 16): consecutive
  // threads read consecutive addresses of the column-major matrices
  double ra[8], rb[8];
  auto load = [&](int st) {
    const int pi = st / per_pair, k0 = (st % per_pair) * kQK;
    // selected by value: a run-time index into the parameter array would copy it to local memory
    const Pair P = pi == 0 ? g.p[0] : pi == 1 ? g.p[1] : g.p[2];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int e = t + q * kQThreads;
      const int ai = e % kQT, ak = e / kQT;
      const int gi = i0 + ai, gk = k0 + ak;
      ra[q] = (gi < d && gk < d) ? P.A[(size_t)gk * d + gi] : 0.0;
      const int bk = e % kQK, bj = e / kQK;
      const int hk = k0 + bk, hj = j0 + bj;
      rb[q] = (hk < d && hj < d) ? P.sign * P.B[(size_t)hj * d + hk] : 0.0;
    }
  };
  if (s0 < s1) load(s0);
  for (int st = s0; st < s1; st++) {
    __syncthreads();   // the previous stage's operands are no longer read
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int e = t + q * kQThreads;
      As[e / kQT][e % kQT] = ra[q];
      Bs[e % kQK][e / kQK] = rb[q];
    }
    __syncthreads();
    if (st + 1 < s1) load(st + 1);   // in flight during this stage's FMAs
#pragma unroll
    for (int k = 0; k < kQK; k++) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        a[q] = As[k][tr * 4 + q];
        b[q] = Bs[k][tc * 4 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; x++)
#pragma unroll
        for (int y = 0; y < 4; y++) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
  }
  if (g.splits == 1) {
#pragma unroll
    for (int y = 0; y < 4; y++) {
      const int j = j0 + tc * 4 + y;
#pragma unroll
      for (int x = 0; x < 4; x++) {
        const int i = i0 + tr * 4 + x;
        if (i < d && j < d) g.C[(size_t)j * d + i] = acc[x][y];
      }
    }
    return;
  }
  // split K: write the partial tile, the last split of the tile sums them in split order
  double* mine = g.part + (size_t)split * d * d;
#pragma unroll
  for (int y = 0; y < 4; y++) {
    const int j = j0 + tc * 4 + y;
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int i = i0 + tr * 4 + x;
      if (i < d && j < d) mine[(size_t)j * d + i] = acc[x][y];
    }
  }
  __threadfence();
  __syncthreads();
  if (t == 0) {
    const unsigned prev = atomicAdd(g.count + tile, 1u);
    last = prev == (unsigned)g.splits - 1;
    if (last) g.count[tile] = 0;   // ready for the next launch
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int y = 0; y < 4; y++) {
    const int j = j0 + tc * 4 + y;
#pragma unroll
    for (int x = 0; x < 4; x++) {
      const int i = i0 + tr * 4 + x;
      if (i < d && j < d) {
        double s = 0.0;
        for (int q = 0; q < g.splits; q++) s += __ldcg(g.part + (size_t)q * d * d + (size_t)j * d + i);
        g.C[(size_t)j * d + i] = s;
      }
    }
  }
}

}  // namespace

int qap_splits(int64_t d, int sms) {
  const int tiles = (int)(((d + kQT - 1) / kQT) * ((d + kQT - 1) / kQT));
  const int stages = (int)((d + kQK - 1) / kQK);   // of one operand pair
  // about two blocks per SM, each split at least four stages of one pair
  int s = (2 * sms + tiles - 1) / tiles;
  s = std::min(s, std::max(1, stages / 4));
  return std::max(1, std::min(s, kQapMaxSplits));
}

cudaError_t qap_apply(const QDev& Q, const double* x, double* out, int splits, cudaStream_t s) {
  const int d = (int)Q.qap_d;
  const double *Ah = Q.qap, *Bh = Q.qap + (size_t)d * d, *S = Q.qap + 2 * (size_t)d * d,
               *T = Q.qap + 3 * (size_t)d * d;
  const int tiles_i = (d + kQT - 1) / kQT;
  const int tiles = tiles_i * tiles_i;
  Gemm g1 = {};
  g1.p[0] = {Ah, x, 1.0};
  g1.npair = 1;
  g1.d = d;
  g1.C = Q.qap_tmp;
  g1.part = Q.qap_part;
  g1.count = Q.qap_count;
  g1.splits = splits;
  k_qap_gemm<<<tiles * splits, kQThreads, 0, s>>>(g1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Gemm g2 = g1;
  g2.p[0] = {Q.qap_tmp, Bh, 1.0};
  g2.p[1] = {S, x, -1.0};
  g2.p[2] = {x, T, -1.0};
  g2.npair = 3;
  g2.C = out;
  k_qap_gemm<<<tiles * splits, kQThreads, 0, s>>>(g2);
  return cudaGetLastError();
}

}  // namespace hprqp
