// hprqp_power_noalloc: the power-method estimate of lambda_A without any device allocation.
//
// Some callers cannot allocate device memory when they need this estimate: real-time loops
// that must not allocate after start-up (an allocation can block on the device or the
// driver), and processes whose device memory is owned entirely by another allocator (a
// framework's pool that leaves nothing for cudaMalloc).  This entry point therefore keeps its
// work vectors, its per-block partial sums and its control scalars in one file-scope device
// array of fixed size; the caller only passes the matrix (and its transpose) and receives the
// estimate.
//
// The array lives in every GPU that loads the library until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress, by the first call on that
// device.  All calls share the array: two calls that overlap on the GPU race with each other.
// Every call initialises the parts it reads (control block, start vector) before using them.
// The call reads the two row-pointer ends and polls the convergence flag with copies to the
// host followed by a synchronisation of its stream, so it cannot run on a stream that is being
// captured into a CUDA graph.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/hprqp.h"
#include "kernels.cuh"

namespace hprqp {
namespace {

constexpr int64_t kNaMaxDim = HPRQP_NOALLOC_MAX_DIM;     // m and n limit
constexpr int kNaMaxGrid = 2048;                        // blocks of one pass
constexpr int64_t kNaCtl = 8;                           // control block (doubles)
constexpr int64_t kNaPart = 2 * kNaMaxGrid;             // partial sums
constexpr int64_t kNaTotal = kNaCtl + kNaPart + 3 * kNaMaxDim;

static __device__ __align__(256) double g_na_scratch[kNaTotal];

// control block layout (doubles): 0 lambda, 1 scale, 2 iteration, 3 state
// (0 running, 2 converged: normalise once more, 1 finished), 4 last-block counter (as unsigned)
struct NaView {
  double* ctl;
  double* part;
  double* v;
  double* w;
  double* tmp;
};

__device__ __forceinline__ unsigned* na_counter(double* ctl) { return reinterpret_cast<unsigned*>(ctl + 4); }

__global__ void k_na_init(NaView s, int64_t m, double scale) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
    // the start vector of the power method in hprqp_solve: 0.5 + (hash(i) mod 2^32) / 2^32
    const uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
    s.w[i] = 0.5 + (double)h / 4294967296.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s.ctl[0] = 0.0;
    s.ctl[1] = scale;
    s.ctl[2] = 0.0;
    s.ctl[3] = 0.0;
    *na_counter(s.ctl) = 0u;
  }
}

// v = w * scale unless finished; a converged state becomes finished afterwards (single block
// flips the state after the grid of the next kernel has read it)
__global__ void k_na_norm(NaView s, int64_t m) {
  if (s.ctl[3] == 1.0) return;
  const double sc = s.ctl[1];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) s.v[i] = s.w[i] * sc;
}
__global__ void k_na_flag(NaView s) {
  if (s.ctl[3] == 2.0) s.ctl[3] = 1.0;
}

// tmp = A^T v  (rows n of the stored transpose)
template <int G>
__global__ void __launch_bounds__(kThreads) k_na_at(NaView s, Csr AT) {
  if (s.ctl[3] != 0.0) return;
  __shared__ double rs0[kChunk];
  const int64_t nchunks = (AT.rows + kChunk - 1) / kChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t row0 = ch * kChunk;
    csr_chunk<G, 1>(AT, row0, s.v, nullptr, rs0, nullptr, false);
    __syncthreads();
    const int64_t j = row0 + threadIdx.x;
    if (j < AT.rows) s.tmp[j] = rs0[threadIdx.x];
    __syncthreads();
  }
}

// w = A tmp, <v, w>, ||w||^2; the last block updates the Rayleigh quotient and the state
template <int G>
__global__ void __launch_bounds__(kThreads) k_na_a(NaView s, Csr A, int64_t max_iter, double tol) {
  if (s.ctl[3] != 0.0) return;
  __shared__ double rs0[kChunk];
  __shared__ double red[kWP * 32];
  double acc[kWP] = {0.0, 0.0};
  const int64_t nchunks = (A.rows + kChunk - 1) / kChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t row0 = ch * kChunk;
    csr_chunk<G, 1>(A, row0, s.tmp, nullptr, rs0, nullptr, false);
    __syncthreads();
    const int64_t j = row0 + threadIdx.x;
    if (j < A.rows) {
      const double wv = rs0[threadIdx.x];
      s.w[j] = wv;
      acc[0] = fma(s.v[j], wv, acc[0]);
      acc[1] = fma(wv, wv, acc[1]);
    }
    __syncthreads();
  }
  block_reduce<kWP>(acc, 0u, red);
  if (threadIdx.x == 0) {
    s.part[(size_t)blockIdx.x * kWP] = acc[0];
    s.part[(size_t)blockIdx.x * kWP + 1] = acc[1];
  }
  if (!last_block(na_counter(s.ctl))) return;
  double tot[kWP];
  reduce_partials<kWP>(s.part, gridDim.x, kWP, 0u, tot, red);
  if (threadIdx.x == 0) {
    const double lnew = tot[0], nw = sqrt(tot[1]);
    if (nw == 0.0 || !isfinite(nw)) {
      s.ctl[0] = 0.0;
      s.ctl[1] = 0.0;
      s.ctl[3] = 1.0;
    } else {
      const double it = s.ctl[2];
      const bool conv = (it > 0.0) && fabs(lnew - s.ctl[0]) <= tol * fabs(lnew);
      s.ctl[0] = lnew;
      s.ctl[1] = 1.0 / nw;
      s.ctl[2] = it + 1.0;
      if (conv || it + 1.0 >= (double)max_iter) s.ctl[3] = 2.0;
    }
  }
}

template <int G>
cudaError_t na_pass(NaView s, const Csr& A, const Csr& AT, int gm, int gn, int ge, int64_t m, int64_t max_iter,
                    double tol, cudaStream_t st) {
  k_na_norm<<<ge, kThreads, 0, st>>>(s, m);
  k_na_flag<<<1, 1, 0, st>>>(s);
  k_na_at<G><<<gn, kThreads, 0, st>>>(s, AT);
  k_na_a<G><<<gm, kThreads, 0, st>>>(s, A, max_iter, tol);
  return cudaGetLastError();
}

std::mutex g_na_mutex;
double* g_na_addr[64] = {nullptr};

}  // namespace
}  // namespace hprqp

using namespace hprqp;

extern "C" hprqp_status hprqp_power_noalloc(int64_t m, int64_t n, const int32_t* A_rowptr, const int32_t* A_colidx,
                                            const double* A_vals, const int32_t* AT_rowptr, const int32_t* AT_colidx,
                                            const double* AT_vals, int64_t max_iter, double tol, double safety,
                                            void* stream, double* lambda_out) {
  if (!lambda_out || m <= 0 || n <= 0 || m > kNaMaxDim || n > kNaMaxDim || max_iter < 1 || !(tol >= 0.0) ||
      !(safety > 0.0) || !A_rowptr || !A_colidx || !A_vals || !AT_rowptr || !AT_colidx || !AT_vals)
    return HPRQP_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return HPRQP_CUDA_ERROR;
  }
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_addr[dev]) {
      // the host-side name of the array is not a device address: look the address up once,
      // with this device current
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HPRQP_CUDA_ERROR;
      }
      g_na_addr[dev] = static_cast<double*>(p);
    }
    base = g_na_addr[dev];
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return HPRQP_CUDA_ERROR;
  }
  // row counts and nnz (host reads of the two row-pointer ends)
  int32_t a_nnz = 0, at_nnz = 0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&a_nnz, A_rowptr + m, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&at_nnz, AT_rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HPRQP_CUDA_ERROR;
  }
  if (a_nnz != at_nnz || a_nnz < 0) return HPRQP_INVALID_ARG;
  Csr A, AT;
  A.rows = m;
  A.cols = n;
  A.nnz = a_nnz;
  A.rp = A_rowptr;
  A.ci = A_colidx;
  A.v = A_vals;
  AT.rows = n;
  AT.cols = m;
  AT.nnz = at_nnz;
  AT.rp = AT_rowptr;
  AT.ci = AT_colidx;
  AT.v = AT_vals;
  NaView s;
  s.ctl = base;
  s.part = base + kNaCtl;
  s.v = base + kNaCtl + kNaPart;
  s.w = s.v + kNaMaxDim;
  s.tmp = s.w + kNaMaxDim;
  auto chunks = [](int64_t rows) { return (int)std::max<int64_t>(1, (rows + kChunk - 1) / kChunk); };
  const int gm = std::min(std::min(chunks(m), sms * 4), kNaMaxGrid);
  const int gn = std::min(std::min(chunks(n), sms * 4), kNaMaxGrid);
  const int ge = std::min(chunks(std::max(m, n)), sms * 8);
  // 1/||start|| in the summation order the CPU reference uses
  double s2 = 0.0;
  for (int64_t i = 0; i < m; i++) {
    const uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
    const double v = 0.5 + (double)h / 4294967296.0;
    s2 += v * v;
  }
  k_na_init<<<ge, kThreads, 0, st>>>(s, m, 1.0 / sqrt(s2));
  const double avg = (double)a_nnz / (double)m;
  const int G = avg < 12 ? 1 : avg < 48 ? 4 : 32;
  double state = 0.0;
  const int64_t chunk = 16;
  // launch rounds of `chunk` steps until the device flag says finished; the kernels stop by
  // themselves after max_iter steps, so max_iter / chunk + 2 rounds always reach that flag
  // (written without max_iter + chunk, which overflows for max_iter near INT64_MAX)
  const int64_t rounds = max_iter / chunk + 2;
  for (int64_t r = 0; r < rounds; r++) {
    for (int64_t i = 0; i < chunk; i++) {
      cudaError_t e = G == 1 ? na_pass<1>(s, A, AT, gm, gn, ge, m, max_iter, tol, st)
                      : G == 4 ? na_pass<4>(s, A, AT, gm, gn, ge, m, max_iter, tol, st)
                               : na_pass<32>(s, A, AT, gm, gn, ge, m, max_iter, tol, st);
      if (e != cudaSuccess) return HPRQP_CUDA_ERROR;
    }
    if (cudaMemcpyAsync(&state, s.ctl + 3, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return HPRQP_CUDA_ERROR;
    }
    if (state == 1.0) break;
  }
  double lam = 0.0;
  if (cudaMemcpyAsync(&lam, s.ctl, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return HPRQP_CUDA_ERROR;
  }
  *lambda_out = safety * lam;
  return HPRQP_OK;
}
