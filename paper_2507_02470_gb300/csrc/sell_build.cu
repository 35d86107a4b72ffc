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


// ---- tiled SELL copies (SellTiles, tiled.cu): per column tile of width W, rows in windows of
// kSellWin sorted by their entry count in the tile (ties by row), slices of 32, 16-bit
// tile-local columns.  Same layout as a host build.

// entry count of every (tile, row): len[k * rows + r] (zeroed beforehand)
__global__ void k_tile_len(const int* __restrict__ rp, const int* __restrict__ ci, int64_t rows, int W,
                           int* __restrict__ len) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += stride)
    for (int q = rp[r]; q < rp[r + 1]; q++) len[(int64_t)(ci[q] / W) * rows + r]++;
}

// block (tile k, window w): rank of each row of the window by decreasing length (ties by
// row); perm[k][position] = row, slot[k * rows + row] = position, width of each slice
__global__ void k_tile_rank(const int* __restrict__ len, int64_t rows, int64_t nsl, int nwin,
                            int* __restrict__ perm, int* __restrict__ slot, int* __restrict__ width) {
  __shared__ int sl[kSellWin];
  const int k = blockIdx.x / nwin, w = blockIdx.x % nwin;
  const int64_t r0 = (int64_t)w * kSellWin;
  const int cnt = (int)(rows - r0 < kSellWin ? rows - r0 : kSellWin);
  const int* lk = len + (int64_t)k * rows;
  for (int t = threadIdx.x; t < kSellWin; t += blockDim.x) sl[t] = t < cnt ? lk[r0 + t] : -1;
  __syncthreads();
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int L = sl[t];
    int rank = 0;
    for (int u = 0; u < cnt; u++) rank += (sl[u] > L) || (sl[u] == L && u < t);
    const int64_t pos = r0 + rank;
    perm[(int64_t)k * nsl * 32 + pos] = (int)(r0 + t);
    slot[(int64_t)k * rows + r0 + t] = (int)pos;
    if (rank % 32 == 0) width[(int64_t)k * nsl + pos / 32] = L;
  }
}

// off[k * (nsl + 1) + s]: entry offset of slice s of tile k, tiles one after the other;
// off[k * (nsl + 1) + nsl]: the running total after tile k; *total: all entries (one block)
__global__ void k_tile_scan(const int* __restrict__ width, int ntile, int64_t nsl, int* __restrict__ off,
                            long long* __restrict__ total) {
  __shared__ long long part[kThreads];
  const int64_t all = (int64_t)ntile * nsl;
  const int t = threadIdx.x;
  const int64_t per = (all + kThreads - 1) / kThreads;
  const int64_t b = t * per, e = b + per < all ? b + per : all;
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
    *total = run;
  }
  __syncthreads();
  long long run = part[t];
  for (int64_t i = b; i < e; i++) {
    const int64_t k = i / nsl, s = i % nsl;
    off[k * (nsl + 1) + s] = (int)run;
    run += 32LL * width[i];
    if (s == nsl - 1) off[k * (nsl + 1) + nsl] = (int)run;
  }
}

// entries of each row into their tile's slice lanes, in row order (col / val zeroed)
__global__ void k_tile_fill(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ v,
                            int64_t rows, int W, int ntile, int64_t nsl, const int* __restrict__ slot,
                            const int* __restrict__ off, unsigned short* __restrict__ col,
                            double* __restrict__ val) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += stride) {
    int m[kMaxTilesDevice];
    for (int k = 0; k < ntile; k++) m[k] = 0;
    for (int q = rp[r]; q < rp[r + 1]; q++) {
      const int k = ci[q] / W;
      const int p = slot[(int64_t)k * rows + r];
      const int64_t pos = (int64_t)off[(int64_t)k * (nsl + 1) + p / 32] + (int64_t)m[k] * 32 + p % 32;
      col[pos] = (unsigned short)(ci[q] - k * W);
      val[pos] = v[q];
      m[k]++;
    }
  }
}

cudaError_t tile_layout(const Csr& M, int W, int ntile, int* len, int* perm, int* slot, int* width, int* off,
                        long long* total, cudaStream_t s) {
  const int64_t rows = M.rows, nsl = (rows + 31) / 32;
  const int nwin = (int)((rows + kSellWin - 1) / kSellWin);
  cudaError_t e = cudaMemsetAsync(len, 0, (size_t)ntile * rows * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(perm, 0xff, (size_t)ntile * nsl * 32 * sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(width, 0, (size_t)ntile * nsl * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<int64_t>((rows + kThreads - 1) / kThreads, 152 * 8);
  k_tile_len<<<blocks, kThreads, 0, s>>>(M.rp, M.ci, rows, W, len);
  k_tile_rank<<<(unsigned)(ntile * nwin), kThreads, 0, s>>>(len, rows, nsl, nwin, perm, slot, width);
  k_tile_scan<<<1, kThreads, 0, s>>>(width, ntile, nsl, off, total);
  return cudaGetLastError();
}

cudaError_t tile_fill(const Csr& M, int W, int ntile, const int* slot, const int* off, unsigned short* col,
                      double* val, cudaStream_t s) {
  const int64_t rows = M.rows, nsl = (rows + 31) / 32;
  const int blocks = (int)std::min<int64_t>((rows + kThreads - 1) / kThreads, 152 * 8);
  k_tile_fill<<<blocks, kThreads, 0, s>>>(M.rp, M.ci, M.v, rows, W, ntile, nsl, slot, off, col, val);
  return cudaGetLastError();
}

// ---- transpose of a CSR matrix on the device, with the layout of the host counting sort
// (entries of each transposed row in increasing original row order)
__global__ void k_tr_count(const int* __restrict__ ci, int64_t nnz, int* __restrict__ cnt) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += stride)
    atomicAdd(cnt + ci[q] + 1, 1);
}

// in-place inclusive scan of rp[0..len) (rp[0] = 0) and the largest difference (one block)
__global__ void k_tr_scan(int* __restrict__ rp, int64_t len, int* __restrict__ maxlen) {
  __shared__ long long part[kThreads];
  __shared__ int mx[kThreads];
  const int t = threadIdx.x;
  const int64_t per = (len + kThreads - 1) / kThreads;
  const int64_t b = t * per, e = b + per < len ? b + per : len;
  long long sum = 0;
  int m = 0;
  for (int64_t i = b; i < e; i++) {
    sum += rp[i];
    m = rp[i] > m ? rp[i] : m;
  }
  part[t] = sum;
  mx[t] = m;
  __syncthreads();
  if (t == 0) {
    long long run = 0;
    int mm = 0;
    for (int i = 0; i < kThreads; i++) {
      const long long v = part[i];
      part[i] = run;
      run += v;
      mm = mx[i] > mm ? mx[i] : mm;
    }
    *maxlen = mm;
  }
  __syncthreads();
  long long run = part[t];
  for (int64_t i = b; i < e; i++) {
    run += rp[i];
    rp[i] = (int)run;
  }
}

// every entry into its column's segment at a free place (any order), keyed by its index q
__global__ void k_tr_fill(const int* __restrict__ ci, const double* __restrict__ v, int64_t nnz,
                          const int* __restrict__ rpT, int* __restrict__ cur, int* __restrict__ ciT,
                          double* __restrict__ vT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += stride) {
    const int c = ci[q];
    const int pos = rpT[c] + atomicAdd(cur + c, 1);
    ciT[pos] = (int)q;
    vT[pos] = v[q];
  }
}

// the entry index q of every place -> its row (binary search in the row pointers)
__global__ void k_tr_rows(const int* __restrict__ rp, int64_t rows, int64_t nnz, int* __restrict__ ciT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz; i += stride) {
    const int q = ciT[i];
    int64_t lo = 0, hi = rows - 1;   // the last row r with rp[r] <= q
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) / 2;
      if (rp[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    ciT[i] = (int)lo;
  }
}

// each transposed row by increasing entry index, i.e. by row and then by place in the row:
// the order of the host counting sort (insertion sort; the keys are distinct)
__global__ void k_tr_sort(const int* __restrict__ rpT, int64_t cols, int* __restrict__ ciT, double* __restrict__ vT) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < cols; c += stride) {
    const int b = rpT[c], e = rpT[c + 1];
    for (int i = b + 1; i < e; i++) {
      const int key = ciT[i];
      const double val = vT[i];
      int j = i - 1;
      while (j >= b && ciT[j] > key) {
        ciT[j + 1] = ciT[j];
        vT[j + 1] = vT[j];
        j--;
      }
      ciT[j + 1] = key;
      vT[j + 1] = val;
    }
  }
}

cudaError_t transpose_layout(const Csr& M, int* rpT, int* maxlen, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(rpT, 0, (size_t)(M.cols + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int blocks = (int)std::min<int64_t>((M.nnz + kThreads - 1) / kThreads + 1, 152 * 8);
  if (M.nnz > 0) k_tr_count<<<blocks, kThreads, 0, s>>>(M.ci, M.nnz, rpT);
  k_tr_scan<<<1, kThreads, 0, s>>>(rpT, M.cols + 1, maxlen);
  return cudaGetLastError();
}

cudaError_t transpose_fill(const Csr& M, const int* rpT, int* cur, int* ciT, double* vT, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(cur, 0, (size_t)(M.cols > 0 ? M.cols : 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  if (M.nnz == 0) return cudaSuccess;
  const int qb = (int)std::min<int64_t>((M.nnz + kThreads - 1) / kThreads + 1, 152 * 8);
  const int cb = (int)std::min<int64_t>((M.cols + kThreads - 1) / kThreads + 1, 152 * 8);
  k_tr_fill<<<qb, kThreads, 0, s>>>(M.ci, M.v, M.nnz, rpT, cur, ciT, vT);
  k_tr_sort<<<cb, kThreads, 0, s>>>(rpT, M.cols, ciT, vT);
  k_tr_rows<<<qb, kThreads, 0, s>>>(M.rp, M.rows, M.nnz, ciT);
  return cudaGetLastError();
}

}  // namespace hprqp
