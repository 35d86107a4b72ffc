// SELL-32 copies of CSR matrices built on the device for the row kernels' SELL schedule
// (csr_chunk_sell): rows sorted by decreasing length inside each 256-row chunk (ties by row),
// slices of 32 rows, entry m of a slice's lane l at off[slice] + 32 m + l, zero-padded to the
// slice's longest row.  Building them here instead of on the host saves the upload.
#include <algorithm>

#include "sell_build.cuh"

namespace hprqp {

// rank of each row inside its 256-row chunk by decreasing length (ties by row): perm[sorted
// position] = row; the width of a slice is the length of its first (longest) row
__global__ void k_sell_rank(const int* __restrict__ rp, int64_t rows, int* __restrict__ perm,
                            int* __restrict__ width) {
  __shared__ int len[kChunk];
  const int64_t r0 = (int64_t)blockIdx.x * kChunk;
  const int t = threadIdx.x;
  const int cnt = (int)(rows - r0 < kChunk ? rows - r0 : kChunk);
  len[t] = t < cnt ? rp[r0 + t + 1] - rp[r0 + t] : -1;
  __syncthreads();
  if (t < cnt) {
    const int L = len[t];
    int rank = 0;
    for (int u = 0; u < cnt; u++) rank += (len[u] > L) || (len[u] == L && u < t);
    perm[r0 + rank] = (int)(r0 + t);
    if (rank % 32 == 0) width[(r0 + rank) / 32] = L;
  }
}

// exclusive prefix sum of 32 * width over the slices into off (one block); *total: the sum
__global__ void k_sell_scan(const int* __restrict__ width, int64_t nsl, int* __restrict__ off,
                            long long* __restrict__ total) {
  __shared__ long long part[kThreads];
  const int t = threadIdx.x;
  const int64_t per = (nsl + kThreads - 1) / kThreads;
  const int64_t b = t * per, e = b + per < nsl ? b + per : nsl;
  long long sum = 0;
  for (int64_t i = b; i < e; i++) sum += 32LL * width[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    for (int i = 0; i < kThreads; i++) {
      const long long v = part[i];
      part[i] = run;
      run += v;
    }
    off[nsl] = (int)run;
    *total = run;
  }
  __syncthreads();
  long long run = part[t];
  for (int64_t i = b; i < e; i++) {
    off[i] = (int)run;
    run += 32LL * width[i];
  }
}

// entries of each row into its lane of its slice (sci / sv zeroed beforehand)
__global__ void k_sell_fill(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                            const int* __restrict__ perm, const int* __restrict__ off, int64_t npos,
                            int* __restrict__ sci, double* __restrict__ sv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npos; p += stride) {
    const int r = perm[p];
    if (r < 0) continue;
    const int64_t base = (int64_t)off[p / 32] + (p % 32);
    for (int q = rp[r]; q < rp[r + 1]; q++) {
      const int64_t pos = base + (int64_t)(q - rp[r]) * 32;
      sci[pos] = ci[q];
      sv[pos] = v[q];
    }
  }
}

cudaError_t sell_layout(const Csr& M, int* perm, int* width, int* off, long long* total, cudaStream_t s) {
  const int64_t nch = (M.rows + kChunk - 1) / kChunk, nsl = (M.rows + 31) / 32;
  cudaError_t e = cudaMemsetAsync(perm, 0xff, (size_t)nsl * 32 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(width, 0, (size_t)nsl * sizeof(int), s);
  if (e != cudaSuccess) return e;
  k_sell_rank<<<(unsigned)nch, kChunk, 0, s>>>(M.rp, M.rows, perm, width);
  k_sell_scan<<<1, kThreads, 0, s>>>(width, nsl, off, total);
  return cudaGetLastError();
}

cudaError_t sell_fill(const Csr& M, const int* perm, const int* off, int* sci, double* sv, cudaStream_t s) {
  const int64_t npos = (M.rows + 31) / 32 * 32;
  const int blocks = (int)std::min<int64_t>((npos + kThreads - 1) / kThreads, 152 * 8);
  k_sell_fill<<<blocks, kThreads, 0, s>>>(M.rp, M.ci, M.v, perm, off, npos, sci, sv);
  return cudaGetLastError();
}

}  // namespace hprqp
