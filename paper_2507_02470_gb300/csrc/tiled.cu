// Shared-memory-tiled products with a factor term B_f (p x n) of Q, for the passes that need
// one vector (every inner step except stopping tests, the restart pass, apply, power method):
//
//   k_tb    partial t_k = B_f[:, tile k] x_k  block (k, g): column tile k of x (kTileW entries)
//                                             in shared memory, share g of the tile's slices
//   k_tsum  t = sum_k t_k                     in tile order (deterministic)
//   k_tbt   u = B_f^T t                       one pass per tile of t: every block holds the tile
//                                             in shared memory and adds its rows' part to u
//
// Why: on GB300 both the FP64 pipe (one warp instruction per 19 cycles per SM) and random
// gathers from L2 (one L1 wavefront per distinct line, about one gather per SM cycle) bound
// these products.  Here each lane owns a row of a 32-row slice (SELL-32 with rows sorted by
// length inside windows of 512): the loads are coalesced, every FMA instruction works on 32
// rows with little padding and no shuffle reduction, and the gathers hit shared memory.
// Padding entries hold the value 0 at column 0: they add 0 * tab[0] (0 for a finite iterate).
// u goes to the intermediate buffer at uoff, where the row pass adds it.
#include "kernels.cuh"

namespace hprqp {

constexpr int kTThreads = 1024;   // threads per tiled block (one block per SM: 200 KB tile)
constexpr size_t kTSmem = (size_t)kTileW * sizeof(double);

namespace {

// Same early exits as the CSR pre-pass; two-vector passes (stopping tests) take the CSR path.
template <int TT>
__device__ __forceinline__ bool tiled_idle(const Ctrl* C, int which) {
  if (pre_in_step(which) && C->done) return true;
  if (which == 2 && !C->restart_pending) return true;
  if (which == 4 && C->pw_done) return true;
  return which == 0 && (TT == 1 || (TT == 2 && C->ttest));
}

// dst[i] = src[i] for i < cnt by the whole block, as asynchronous 8-byte copies (all in flight
// at once; a load-then-store loop would wait for each load in turn); completes with a barrier
__device__ __forceinline__ void tile_copy(double* dst, const double* src, int cnt) {
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + i);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

// This lane's row of the slice whose entries are [b, e) (e - b a multiple of 32): the sum of
// val * tab[col] over its entries in order.  Software-pipelined: the loads of the next four
// entries are issued before the products of the current four (a warp issues in order, so
// otherwise it would wait for each group's loads only after finishing the previous products).
__device__ __forceinline__ double sell_row(int b, int e, int lane, const unsigned short* __restrict__ col,
                                           const double* __restrict__ val, const double* tab) {
  constexpr int U = 4;
  double acc = 0.0;
  int q = b + lane;
  unsigned c[U];
  double v[U];
#pragma unroll
  for (int u = 0; u < U; u++) {
    const bool h = q + u * kSellC < e;
    c[u] = h ? col[q + u * kSellC] : 0u;
    v[u] = h ? val[q + u * kSellC] : 0.0;
  }
  while (q < e) {
    const int qn = q + U * kSellC;
    unsigned cn[U];
    double vn[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const bool h = qn + u * kSellC < e;
      cn[u] = h ? col[qn + u * kSellC] : 0u;
      vn[u] = h ? val[qn + u * kSellC] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; u++)
      if (q + u * kSellC < e) acc = fma(v[u], tab[c[u]], acc);
#pragma unroll
    for (int u = 0; u < U; u++) {
      c[u] = cn[u];
      v[u] = vn[u];
    }
    q = qn;
  }
  return acc;
}

// The slices [s0, s1) of one tile, shared among the warps of the block: round i gives warp w
// slice s0 + 32 i + (w + i) mod 32 (inside a window the slices run from the longest rows to
// the shortest, so the rotation gives every warp long and short slices).  For each lane's row:
// out(row, sum, pre(row)), where pre(row) (a load the output needs) is issued together with
// the next slice's bounds and row, before the current slice's entries.
template <typename Pre, typename Out>
__device__ __forceinline__ void sell_slices(const int* off, const int* perm, const unsigned short* col,
                                            const double* val, int64_t s0, int64_t s1, const double* tab,
                                            Pre pre, Out out) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  auto slice = [&](int64_t i) { return s0 + i * 32 + (warp + i) % 32; };
  const int64_t rounds = (s1 - s0 + 31) / 32;
  int nb = 0, ne = 0, nrow = -1;
  double npre = 0.0;
  if (rounds > 0 && slice(0) < s1) {
    nb = off[slice(0)];
    ne = off[slice(0) + 1];
    nrow = perm[slice(0) * kSellC + lane];
    if (nrow >= 0) npre = pre(nrow);
  }
  for (int64_t i = 0; i < rounds; i++) {
    if (slice(i) >= s1) continue;   // the same for the whole warp
    const int b = nb, e = ne, row = nrow;
    const double rpre = npre;
    if (i + 1 < rounds && slice(i + 1) < s1) {
      const int64_t sl = slice(i + 1);
      nb = off[sl];
      ne = off[sl + 1];
      nrow = perm[sl * kSellC + lane];
      if (nrow >= 0) npre = pre(nrow);
    }
    const double acc = sell_row(b, e, lane, col, val, tab);
    if (row >= 0) out(row, acc, rpre);
  }
}

template <int TT>
__global__ void __launch_bounds__(kTThreads, 1) k_tb(Args a, int which, int f) {
  pdl_enter();
  if (tiled_idle<TT>(a.C, which)) return;
  extern __shared__ double sx[];
  const TiledFac& T = a.Q.tf[f];
  const SellTiles& M = T.b;
  const Vec& V = a.V;
  const int64_t n = a.n, p = T.p;
  const int k = (int)(blockIdx.x % (unsigned)M.ntile), g = (int)(blockIdx.x / (unsigned)M.ntile);
  const int64_t c0 = (int64_t)k * kTileW;
  const int cw = (int)(n - c0 < (int64_t)kTileW ? n - c0 : (int64_t)kTileW);
  const double* x0 = which == PRE_WH ? (a.m > 0 ? V.wh : V.wb) : which == PRE_WB ? V.wb : which == PRE_AIN ? V.ain
                     : which == PRE_W ? V.w : V.pv;
  if (which == 2) {   // restart: the difference of two vectors
    for (int i = threadIdx.x; i < cw; i += blockDim.x) sx[i] = V.ATyb[c0 + i] - V.ATy0[c0 + i];
    __syncthreads();
  } else {
    tile_copy(sx, x0 + c0, cw);
  }
  // this block's share of the tile's slices
  const int64_t s0 = (int64_t)g * M.nsl / T.nrange, s1 = (int64_t)(g + 1) * M.nsl / T.nrange;
  const int* off = M.off + (size_t)k * (size_t)(M.nsl + 1);
  const int* perm = M.perm + (size_t)k * (size_t)M.nsl * kSellC;
  double* part = T.part + (size_t)k * (size_t)p;
  sell_slices(off, perm, M.col, M.val, s0, s1, sx, [](int) { return 0.0; },
              [&](int row, double acc, double) { part[row] = acc; });
}

// t = sum of the tiles' partial sums, in tile order
template <int TT>
__global__ void __launch_bounds__(kThreads) k_tsum(Args a, int which, int f) {
  pdl_enter();
  if (tiled_idle<TT>(a.C, which)) return;
  const TiledFac& T = a.Q.tf[f];
  const int64_t p = T.p;
  const int kb = T.b.ntile;
  double* t = (pre_into_t1(which) ? a.V.t1 : a.V.t2) + a.Q.toff[f];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < p; r += stride) {
    double s = 0.0;
    int k = 0;
    for (; k + 7 < kb; k += 8) {
      double q[8];
#pragma unroll
      for (int u = 0; u < 8; u++) q[u] = T.part[(size_t)(k + u) * p + r];
#pragma unroll
      for (int u = 0; u < 8; u++) s += q[u];
    }
    for (; k < kb; k++) s += T.part[(size_t)k * p + r];
    t[r] = s;
  }
}

// u = B^T t, tile by tile of t: u = (tile 0 part), then u += (tile k part)
template <int TT>
__global__ void __launch_bounds__(kTThreads, 1) k_tbt(Args a, int which, int f) {
  pdl_enter();
  if (tiled_idle<TT>(a.C, which)) return;
  extern __shared__ double st[];
  const TiledFac& T = a.Q.tf[f];
  const SellTiles& M = T.bt;
  const Vec& V = a.V;
  const int64_t p = T.p;
  double* tb = pre_into_t1(which) ? V.t1 : V.t2;
  const double* tv = tb + a.Q.toff[f];
  double* u = tb + a.Q.uoff[f];
  // this block's share: whole windows (a window holds the same rows in every tile, sorted
  // differently), so u of the previous tile was written by this block
  constexpr int spw = kSellWin / kSellC;
  const int64_t nwin = (M.nsl + spw - 1) / spw;
  const int64_t w0 = (int64_t)blockIdx.x * nwin / gridDim.x, w1 = (int64_t)(blockIdx.x + 1) * nwin / gridDim.x;
  const int64_t s0 = w0 * spw, s1 = w1 * spw < M.nsl ? w1 * spw : M.nsl;
  for (int k = 0; k < M.ntile; k++) {
    const int64_t c0 = (int64_t)k * kTileW;
    const int cw = (int)(p - c0 < (int64_t)kTileW ? p - c0 : (int64_t)kTileW);
    // the previous tile is no longer read, and u of the previous tile is visible to the block
    __syncthreads();
    tile_copy(st, tv + c0, cw);
    const int* off = M.off + (size_t)k * (size_t)(M.nsl + 1);
    const int* perm = M.perm + (size_t)k * (size_t)M.nsl * kSellC;
    const bool first = k == 0;
    sell_slices(off, perm, M.col, M.val, s0, s1, st, [&](int j) { return first ? 0.0 : u[j]; },
                [&](int j, double acc, double prev) { u[j] = first ? acc : prev + acc; });
  }
}

using TiledKernel = void (*)(Args, int, int);
TiledKernel tb_kernel(int tt) { return tt == 0 ? k_tb<0> : tt == 1 ? k_tb<1> : k_tb<2>; }
TiledKernel tsum_kernel(int tt) { return tt == 0 ? k_tsum<0> : tt == 1 ? k_tsum<1> : k_tsum<2>; }
TiledKernel tbt_kernel(int tt) { return tt == 0 ? k_tbt<0> : tt == 1 ? k_tbt<1> : k_tbt<2>; }

}  // namespace

cudaError_t tiled_setup() {
  for (int tt = 0; tt < 3; tt++) {
    cudaError_t e = cudaFuncSetAttribute((const void*)tb_kernel(tt), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void*)tbt_kernel(tt), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTSmem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int tiled_tbt_grid(int64_t n, int sms) {
  const int64_t windows = (n + kSellWin - 1) / kSellWin;
  return (int)(windows < sms ? windows : sms);
}

// t = B_f x (and, except for the restart pass, u = B_f^T t) for every tiled factor term
cudaError_t launch_tiled(const Args& a, const Plan& p, int which, int tt, cudaStream_t s, int* launched) {
  int cnt = 0;
  for (int f = 0; f < a.Q.nfac; f++) {
    if (!a.Q.tiled[f]) continue;
    const TiledFac& T = a.Q.tf[f];
    tb_kernel(tt)<<<T.b.ntile * T.nrange, kTThreads, kTSmem, s>>>(a, which, f);
    const int64_t sb = (T.p + kThreads - 1) / kThreads;
    tsum_kernel(tt)<<<(int)(sb < 152 * 8 ? sb : 152 * 8), kThreads, 0, s>>>(a, which, f);
    cnt += 2;
    if (which != 2) {
      tbt_kernel(tt)<<<p.gridT, kTThreads, kTSmem, s>>>(a, which, f);
      cnt++;
    }
  }
  if (launched) *launched = cnt;
  return cudaGetLastError();
}

}  // namespace hprqp
