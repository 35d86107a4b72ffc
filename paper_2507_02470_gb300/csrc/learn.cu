// Learned warm start: conversions, the BF16 multilayer perceptron (forward, backward, Adam),
// the warm-start loss and the decoder.  Every dense product goes through the tcgen05 GEMM of
// tc_gemm.cu in the single form C = A B^T (both operands K-major); the kernels here are the
// elementwise and transposing steps around those products.
//
// Layouts.  A batch of B instances is kept in two layouts: batch-major (B x d, one instance
// per row) and feature-major (d x B, one feature per row, leading dimension ldT).  With W the
// dout x din weight matrix (row-major) and W^T its transposed copy:
//   forward   acc (dout x B)  = W   * X^T        A = W      (dout x din), B = X      (B x din)
//   weights   dW  (dout x din) = dZ^T * X        A = dZ^T   (dout x B),   B = X^T    (din x B)
//   inputs    dX^T (din x B)   = W^T * dZ^T      A = W^T    (din x dout), B = dZ     (B x dout)
// so each layer stores its BF16 input in both layouts and each gradient dZ in both layouts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hprqp_learn.h"
#include "tc_gemm.cuh"

namespace {

thread_local std::string g_err;

hprqp_status lfail(hprqp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define LCU(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return lfail(e_ == cudaErrorMemoryAllocation ? HPRQP_OOM : HPRQP_CUDA_ERROR, "%s: %s", \
                   #call, cudaGetErrorString(e_));                                           \
  } while (0)

inline int64_t round8(int64_t x) { return (x + 7) / 8 * 8; }

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

hprqp_status gemm(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb,
                  float* C, int64_t ldc, int splits, float* work, cudaStream_t s) {
  const char* why = nullptr;
  cudaError_t e = hprqp::tc::gemm_bf16(M, N, K, A, lda, B, ldb, C, ldc, splits, work, s, &why);
  if (e == cudaErrorInvalidValue && why) return lfail(HPRQP_INVALID_ARG, "gemm: %s", why);
  if (e != cudaSuccess) return lfail(HPRQP_CUDA_ERROR, "gemm: %s", cudaGetErrorString(e));
  return HPRQP_OK;
}

// K-splits that fill the GPU with about one wave of CTAs without exceeding the work buffer
int pick_splits(int64_t M, int64_t N, int64_t K, int64_t work_floats, int sms) {
  const int64_t tiles = ((M + 127) / 128) * ((N + 127) / 128);
  const int64_t kb = (K + 63) / 64;
  int64_t s = std::max<int64_t>(1, sms / std::max<int64_t>(tiles, 1));
  s = std::min(s, kb);
  if (s > 1) s = std::min(s, work_floats / std::max<int64_t>(M * N, 1));
  return (int)std::max<int64_t>(1, s);
}

int device_sms() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// ------------------------------------------------------------------------ conversions
__device__ __forceinline__ uint16_t to_bf16(double v) {
  if (!isfinite(v)) v = 0.0;
  return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));
}
__device__ __forceinline__ uint16_t f_to_bf16(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

template <int NT>
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < NT / 32; ++i) t += red[i];
  return t;   // valid in thread 0
}

// one block per row: out = bf16((x - sub) * scale), padding zeroed, optional FP64 row norm^2
template <typename T>
__global__ void __launch_bounds__(256) k_cast(const T* __restrict__ x, int64_t rows, int64_t cols, int64_t ldx,
                                              const double* __restrict__ sub, double scale, uint16_t* __restrict__ out,
                                              int64_t ldo, double* __restrict__ rownorm2) {
  __shared__ double red[8];
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < ldo; j += 256) {
      uint16_t o = 0;
      if (j < cols) {
        double v = (double)x[i * ldx + j];
        if (sub) v -= sub[j];
        v *= scale;
        if (isfinite(v)) acc += v * v;
        o = to_bf16(v);
      }
      out[i * ldo + j] = o;
    }
    if (rownorm2) {
      const double t = block_sum<256>(acc, red);
      if (threadIdx.x == 0) rownorm2[i] = t;
    }
  }
}

__global__ void __launch_bounds__(256) k_row_stats(const float* __restrict__ F, int64_t rows, int64_t cols, int64_t ld,
                                                   float floor_, float* __restrict__ mean, float* __restrict__ istd) {
  __shared__ double red[8];
  __shared__ double mu_s;
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    double s = 0.0;
    for (int64_t j = threadIdx.x; j < cols; j += 256) s += (double)F[i * ld + j];
    double t = block_sum<256>(s, red);
    if (threadIdx.x == 0) mu_s = t / (double)cols;
    __syncthreads();
    const double mu = mu_s;
    double q = 0.0;
    for (int64_t j = threadIdx.x; j < cols; j += 256) {
      const double d = (double)F[i * ld + j] - mu;
      q += d * d;
    }
    t = block_sum<256>(q, red);
    if (threadIdx.x == 0) {
      mean[i] = (float)mu;
      istd[i] = (float)(1.0 / sqrt(fmax(t / (double)cols, (double)floor_)));
    }
    __syncthreads();
  }
}

__global__ void k_col_mean(const double* __restrict__ Z, int64_t rows, int64_t cols, int64_t ld,
                           double* __restrict__ mu) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cols; j += stride) {
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i) s += Z[i * ld + j];
    mu[j] = s / (double)rows;
  }
}

// ------------------------------------------------------------------------ transposing epilogues
// 32 x 32 tiles through shared memory; block (32, 8).
enum EpiMode { EPI_HIDDEN = 0, EPI_FINAL = 1, EPI_MASK = 2, EPI_STD = 3 };

// Source: FP32 feature-major acc (R x B, ldacc).
//   HIDDEN: v = bf16(relu(acc + bias))  -> outT (R x ldT), outB (B x ldB)
//   FINAL:  Y[b][j] = acc + bias        (FP32 batch-major)
//   MASK:   v = bf16(acc * [mask > 0])  -> outT, outB   (mask: BF16 feature-major, ldmask)
//   STD:    v = bf16((acc - bias) * scl) -> outB only   (feature standardisation)
template <int MODE>
__global__ void k_epi(const float* __restrict__ acc, int64_t ldacc, int R, int B, const float* __restrict__ bias,
                      const float* __restrict__ scl, const uint16_t* __restrict__ mask, int64_t ldmask,
                      uint16_t* __restrict__ outB, int64_t ldB, uint16_t* __restrict__ outT, int64_t ldT,
                      float* __restrict__ Y, int64_t ldy) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int j = j0 + jj, b = b0 + threadIdx.x;
    float v = 0.f;
    if (j < R && b < B) {
      v = acc[(int64_t)j * ldacc + b];
      if (MODE == EPI_HIDDEN || MODE == EPI_FINAL) v += bias[j];
      if (MODE == EPI_HIDDEN) v = fmaxf(v, 0.f);
      if (MODE == EPI_MASK) v = bf16_to_f(mask[(int64_t)j * ldmask + b]) > 0.f ? v : 0.f;
      if (MODE == EPI_STD) v = (v - bias[j]) * scl[j];
      if (MODE != EPI_FINAL) {
        const uint16_t h = f_to_bf16(v);
        v = bf16_to_f(h);
        if (MODE != EPI_STD) outT[(int64_t)j * ldT + b] = h;
      }
    }
    tile[jj][threadIdx.x] = v;
  }
  __syncthreads();
  for (int bb = threadIdx.y; bb < 32; bb += 8) {
    const int b = b0 + bb, j = j0 + threadIdx.x;
    if (b < B && j < R) {
      const float v = tile[threadIdx.x][bb];
      if (MODE == EPI_FINAL) Y[(int64_t)b * ldy + j] = v;
      else outB[(int64_t)b * ldB + j] = f_to_bf16(v);
    }
  }
}

// Source: batch-major FP32 (B x R, ld) -> BF16 batch-major outB and feature-major outT
__global__ void k_from_batch_f32(const float* __restrict__ src, int64_t ld, int R, int B, uint16_t* __restrict__ outB,
                                 int64_t ldB, uint16_t* __restrict__ outT, int64_t ldT) {
  __shared__ uint16_t tile[32][34];
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  for (int bb = threadIdx.y; bb < 32; bb += 8) {
    const int b = b0 + bb, j = j0 + threadIdx.x;
    uint16_t h = 0;
    if (b < B && j < R) {
      h = f_to_bf16(src[(int64_t)b * ld + j]);
      outB[(int64_t)b * ldB + j] = h;
    }
    tile[bb][threadIdx.x] = h;
  }
  __syncthreads();
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int j = j0 + jj, b = b0 + threadIdx.x;
    if (b < B && j < R) outT[(int64_t)j * ldT + b] = tile[threadIdx.x][jj];
  }
}

// BF16 batch-major (B x R, ld) -> feature-major (R x ldT)
__global__ void k_transpose_bf16(const uint16_t* __restrict__ src, int64_t ld, int R, int B, uint16_t* __restrict__ outT,
                                 int64_t ldT) {
  __shared__ uint16_t tile[32][34];
  const int j0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
  for (int bb = threadIdx.y; bb < 32; bb += 8) {
    const int b = b0 + bb, j = j0 + threadIdx.x;
    tile[bb][threadIdx.x] = (b < B && j < R) ? src[(int64_t)b * ld + j] : (uint16_t)0;
  }
  __syncthreads();
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int j = j0 + jj, b = b0 + threadIdx.x;
    if (b < B && j < R) outT[(int64_t)j * ldT + b] = tile[threadIdx.x][jj];
  }
}

// db[j] = sum_b dzT[j][b] (BF16 values, FP64 accumulation in a fixed order)
__global__ void __launch_bounds__(256) k_rowsum_bf16(const uint16_t* __restrict__ dzT, int64_t ldT, int R, int B,
                                                     float* __restrict__ db) {
  __shared__ double red[8];
  for (int j = blockIdx.x; j < R; j += gridDim.x) {
    double s = 0.0;
    for (int b = threadIdx.x; b < B; b += 256) s += (double)bf16_to_f(dzT[(int64_t)j * ldT + b]);
    const double t = block_sum<256>(s, red);
    if (threadIdx.x == 0) db[j] = (float)t;
    __syncthreads();
  }
}

// Adam on a dout x din weight (tiles of 32 x 32, block (32, 8)) refreshing W (BF16, ldw) and
// W^T (BF16, ldwt); `step` = 0 only refreshes the BF16 copies.
__global__ void k_adam_w(float* __restrict__ W, float* __restrict__ mW, float* __restrict__ vW,
                         const float* __restrict__ g, int dout, int din, int step, float lr, float b1, float b2,
                         float eps, float bc1, float bc2, uint16_t* __restrict__ Wb, int64_t ldw,
                         uint16_t* __restrict__ WbT, int64_t ldwt) {
  __shared__ uint16_t tile[32][34];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;   // i: input index (column), j: output row
  for (int jj = threadIdx.y; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + threadIdx.x;
    uint16_t h = 0;
    if (j < dout && i < din) {
      const int64_t e = (int64_t)j * din + i;
      float w = W[e];
      if (step) {
        const float gi = g[e];
        const float m = b1 * mW[e] + (1.f - b1) * gi;
        const float v = b2 * vW[e] + (1.f - b2) * gi * gi;
        mW[e] = m;
        vW[e] = v;
        w -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
        W[e] = w;
      }
      h = f_to_bf16(w);
      Wb[(int64_t)j * ldw + i] = h;
    }
    tile[jj][threadIdx.x] = h;
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + threadIdx.x;
    if (i < din && j < dout) WbT[(int64_t)i * ldwt + j] = tile[threadIdx.x][ii];
  }
}

__global__ void k_adam_b(float* __restrict__ b, float* __restrict__ mb, float* __restrict__ vb,
                         const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float bc1,
                         float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float m = b1 * mb[i] + (1.f - b1) * gi;
  const float v = b2 * vb[i] + (1.f - b2) * gi * gi;
  mb[i] = m;
  vb[i] = v;
  b[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
}

// ------------------------------------------------------------------------ warm-start loss
// One block per instance b: (G o)_k for the latent o = O[b][1..r], the gradient, and the two
// loss parts of the instance (written to part[2b], part[2b+1]).
__global__ void __launch_bounds__(256) k_ws_loss(const float* __restrict__ O, int64_t ldo, int B, int r,
                                                 const float* __restrict__ G, const float* __restrict__ R, int64_t ldr,
                                                 const double* __restrict__ dd, const float* __restrict__ s,
                                                 float s_mean, float s_istd, float alpha, float E, float w_sigma,
                                                 float* __restrict__ dO, int64_t lddo, int out_cols,
                                                 double* __restrict__ part) {
  extern __shared__ float o_s[];
  __shared__ double red[8];
  const int b = blockIdx.x;
  for (int k = threadIdx.x; k < r; k += 256) o_s[k] = O[(int64_t)b * ldo + 1 + k];
  __syncthreads();
  const float invB = 1.f / (float)B;
  double quad = 0.0, lin = 0.0;
  for (int k = threadIdx.x; k < r; k += 256) {
    float go = 0.f;
    for (int j = 0; j < r; ++j) go += G[(int64_t)k * r + j] * o_s[j];
    const float rk = R[(int64_t)k * ldr + b];
    dO[(int64_t)b * lddo + 1 + k] = (alpha * alpha * go - alpha * rk) / E * invB;
    quad += (double)o_s[k] * (double)go;
    lin += (double)o_s[k] * (double)rk;
  }
  for (int k = 1 + r + threadIdx.x; k < out_cols; k += 256) dO[(int64_t)b * lddo + k] = 0.f;
  const double q = block_sum<256>(quad, red);
  const double l = block_sum<256>(lin, red);
  if (threadIdx.x == 0) {
    const float e0 = O[(int64_t)b * ldo] - (s[b] - s_mean) * s_istd;
    dO[(int64_t)b * lddo] = w_sigma * e0 * invB;
    part[2 * b] = 0.5 * (double)w_sigma * (double)e0 * (double)e0;
    part[2 * b + 1] = 0.5 * ((double)alpha * alpha * q - 2.0 * (double)alpha * l + dd[b]) / (double)E;
  }
}

__global__ void k_ws_loss_sum(const double* __restrict__ part, int B, float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, c = 0.0;
  for (int b = 0; b < B; ++b) {
    a += part[2 * b];
    c += part[2 * b + 1];
  }
  loss[0] = (float)(a / B);
  loss[1] = (float)(c / B);
}

// Z[b][i] = clip(mu[i] + alpha work[i][b], lo[i], hi[i]), work feature-major (D x B)
__global__ void k_decode(const float* __restrict__ work, int64_t D, int B, float alpha, const double* __restrict__ mu,
                         const double* __restrict__ lo, const double* __restrict__ hi, double* __restrict__ Z,
                         int64_t ldz) {
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int b0 = blockIdx.y * 32;
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int64_t i = i0 + ii;
    const int b = b0 + threadIdx.x;
    tile[ii][threadIdx.x] = (i < D && b < B) ? work[i * B + b] : 0.f;
  }
  __syncthreads();
  for (int bb = threadIdx.y; bb < 32; bb += 8) {
    const int b = b0 + bb;
    const int64_t i = i0 + threadIdx.x;
    if (b < B && i < D) {
      double z = mu[i] + (double)alpha * (double)tile[threadIdx.x][bb];
      z = fmin(fmax(z, lo[i]), hi[i]);
      Z[(int64_t)b * ldz + i] = z;
    }
  }
}

__global__ void k_sigma0(const float* __restrict__ O, int64_t ldo, int B, float s_mean, float s_istd,
                         double* __restrict__ sigma0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) sigma0[b] = exp((double)s_mean + (double)O[(int64_t)b * ldo] / (double)s_istd);
}

}  // namespace

// ==================================================================================== C ABI
extern "C" const char* hprqp_learn_last_error(void) { return g_err.c_str(); }

extern "C" hprqp_status hprqp_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                                        const uint16_t* B, int64_t ldb, float* C, int64_t ldc, int32_t splits,
                                        float* work, void* stream) {
  return gemm(M, N, K, A, lda, B, ldb, C, ldc, splits, work, (cudaStream_t)stream);
}

extern "C" hprqp_status hprqp_learn_check(void) {
  const int f = hprqp::tc::gemm_error_flag();
  if (f < 0) return lfail(HPRQP_CUDA_ERROR, "could not read the GEMM error flag");
  if (f > 0) return lfail(HPRQP_TIMEOUT, "a GEMM kernel gave up a bounded wait (role %d)", f);
  return HPRQP_OK;
}

template <typename T>
static hprqp_status cast_impl(const T* x, int64_t rows, int64_t cols, int64_t ldx, const double* sub, double scale,
                              uint16_t* out, int64_t ldo, double* rownorm2, void* stream) {
  if (rows < 0 || cols < 0 || ldx < cols || ldo < cols) return lfail(HPRQP_INVALID_ARG, "cast: bad sizes");
  if (rows == 0 || ldo == 0) return HPRQP_OK;
  if (!x || !out) return lfail(HPRQP_INVALID_ARG, "cast: null pointer");
  const int blocks = (int)std::min<int64_t>(rows, 65535);
  k_cast<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(x, rows, cols, ldx, sub, scale, out, ldo, rownorm2);
  LCU(cudaGetLastError());
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_cast_bf16_f64(const double* x, int64_t rows, int64_t cols, int64_t ldx,
                                            const double* sub, double scale, uint16_t* out, int64_t ldo,
                                            double* rownorm2, void* stream) {
  return cast_impl(x, rows, cols, ldx, sub, scale, out, ldo, rownorm2, stream);
}

extern "C" hprqp_status hprqp_cast_bf16_f32(const float* x, int64_t rows, int64_t cols, int64_t ldx,
                                            const double* sub, double scale, uint16_t* out, int64_t ldo,
                                            double* rownorm2, void* stream) {
  return cast_impl(x, rows, cols, ldx, sub, scale, out, ldo, rownorm2, stream);
}

extern "C" hprqp_status hprqp_row_stats(const float* F, int64_t rows, int64_t cols, int64_t ld, float floor_,
                                        float* mean, float* istd, void* stream) {
  if (rows < 0 || cols < 1 || ld < cols) return lfail(HPRQP_INVALID_ARG, "row_stats: bad sizes");
  if (rows == 0) return HPRQP_OK;
  if (!F || !mean || !istd) return lfail(HPRQP_INVALID_ARG, "row_stats: null pointer");
  k_row_stats<<<(int)std::min<int64_t>(rows, 65535), 256, 0, (cudaStream_t)stream>>>(F, rows, cols, ld, floor_, mean,
                                                                                       istd);
  LCU(cudaGetLastError());
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_col_mean_f64(const double* Z, int64_t rows, int64_t cols, int64_t ld, double* mu,
                                           void* stream) {
  if (rows < 1 || cols < 0 || ld < cols) return lfail(HPRQP_INVALID_ARG, "col_mean: bad sizes");
  if (cols == 0) return HPRQP_OK;
  if (!Z || !mu) return lfail(HPRQP_INVALID_ARG, "col_mean: null pointer");
  const int blocks = (int)std::min<int64_t>((cols + 255) / 256, 65535);
  k_col_mean<<<blocks, 256, 0, (cudaStream_t)stream>>>(Z, rows, cols, ld, mu);
  LCU(cudaGetLastError());
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_ws_standardize(const float* F, int64_t d, int64_t B, int64_t ldf, const float* mean,
                                             const float* istd, uint16_t* X, int64_t ldx, void* stream) {
  if (d < 1 || B < 0 || ldf < B || ldx < d || d > (1 << 30) || B > (1 << 30))
    return lfail(HPRQP_INVALID_ARG, "standardize: bad sizes");
  if (B == 0) return HPRQP_OK;
  if (!F || !mean || !istd || !X) return lfail(HPRQP_INVALID_ARG, "standardize: null pointer");
  dim3 grid((unsigned)((B + 31) / 32), (unsigned)((d + 31) / 32));
  if (grid.y > 65535) return lfail(HPRQP_INVALID_ARG, "standardize: d too large");
  k_epi<EPI_STD><<<grid, dim3(32, 8), 0, (cudaStream_t)stream>>>(F, ldf, (int)d, (int)B, mean, istd, nullptr, 0, X,
                                                                  ldx, nullptr, 0, nullptr, 0);
  LCU(cudaGetLastError());
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ MLP
struct MlpLayer {
  int din = 0, dout = 0;
  int64_t ldw = 0, ldwt = 0;   // BF16 W (dout x ldw), W^T (din x ldwt)
  float *W = nullptr, *b = nullptr, *gW = nullptr, *gb = nullptr;
  float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
  uint16_t *Wb = nullptr, *WbT = nullptr;
};

struct hprqp_mlp {
  int L = 0;
  std::vector<int> dims;
  int maxB = 0;
  int64_t ldT = 0;                   // leading dimension of feature-major arrays
  cudaStream_t s = nullptr;
  std::vector<MlpLayer> layers;
  std::vector<uint16_t*> actB, actT;  // input of layer l: batch-major (maxB x round8(d_l)), feature-major
  std::vector<uint16_t*> dzB, dzT;    // gradient w.r.t. the output of layer l (before ReLU)
  float* acc = nullptr;              // FP32 feature-major product (max d x ldT)
  float* work = nullptr;             // split-K partials
  int64_t work_floats = 0;
  int B = 0;                         // batch of the last forward
  int sms = 148;
  std::vector<void*> allocs;
};

static hprqp_status mlp_alloc(hprqp_mlp* n, void** p, size_t bytes) {
  LCU(cudaMalloc(p, std::max<size_t>(bytes, 256)));
  n->allocs.push_back(*p);
  LCU(cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 256), n->s));
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_destroy(hprqp_mlp* net) {
  if (!net) return HPRQP_OK;
  cudaStreamSynchronize(net->s);
  for (void* p : net->allocs) cudaFree(p);
  delete net;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_create(hprqp_mlp** out, int32_t nlayers, const int32_t* dims, int32_t max_batch,
                                         void* stream) {
  if (!out) return lfail(HPRQP_INVALID_ARG, "mlp_create: null output");
  *out = nullptr;
  if (nlayers < 1 || nlayers > 16 || !dims || max_batch < 1 || max_batch > (1 << 20))
    return lfail(HPRQP_INVALID_ARG, "mlp_create: need 1..16 layers, dims, 1 <= max_batch <= 2^20");
  for (int l = 0; l <= nlayers; ++l)
    if (dims[l] < 1 || dims[l] > (1 << 16)) return lfail(HPRQP_INVALID_ARG, "mlp_create: width %d out of range", dims[l]);
  hprqp_mlp* n = new hprqp_mlp();
  n->L = nlayers;
  n->dims.assign(dims, dims + nlayers + 1);
  n->maxB = max_batch;
  n->ldT = round8(max_batch);
  n->s = (cudaStream_t)stream;
  n->sms = device_sms();
  hprqp_status st;
  auto A = [&](void* pp, size_t bytes) { return mlp_alloc(n, reinterpret_cast<void**>(pp), bytes); };
  n->layers.resize(nlayers);
  int dmax = 0;
  for (int l = 0; l <= nlayers; ++l) dmax = std::max(dmax, dims[l]);
  for (int l = 0; l < nlayers; ++l) {
    MlpLayer& y = n->layers[l];
    y.din = dims[l];
    y.dout = dims[l + 1];
    y.ldw = round8(y.din);
    y.ldwt = round8(y.dout);
    const size_t nw = (size_t)y.din * y.dout;
    if ((st = A(&y.W, nw * 4)) || (st = A(&y.gW, nw * 4)) || (st = A(&y.mW, nw * 4)) || (st = A(&y.vW, nw * 4)) ||
        (st = A(&y.b, y.dout * 4)) || (st = A(&y.gb, y.dout * 4)) || (st = A(&y.mb, y.dout * 4)) ||
        (st = A(&y.vb, y.dout * 4)) || (st = A(&y.Wb, (size_t)y.dout * y.ldw * 2)) ||
        (st = A(&y.WbT, (size_t)y.din * y.ldwt * 2))) {
      hprqp_mlp_destroy(n);
      return st;
    }
  }
  n->actB.assign(nlayers, nullptr);
  n->actT.assign(nlayers, nullptr);
  n->dzB.assign(nlayers, nullptr);
  n->dzT.assign(nlayers, nullptr);
  for (int l = 0; l < nlayers; ++l) {
    if ((st = A(&n->actB[l], (size_t)max_batch * round8(dims[l]) * 2)) ||
        (st = A(&n->actT[l], (size_t)dims[l] * n->ldT * 2)) ||
        (st = A(&n->dzB[l], (size_t)max_batch * round8(dims[l + 1]) * 2)) ||
        (st = A(&n->dzT[l], (size_t)dims[l + 1] * n->ldT * 2))) {
      hprqp_mlp_destroy(n);
      return st;
    }
  }
  n->work_floats = std::max<int64_t>((int64_t)n->sms * 128 * 128, (int64_t)dmax * 8);
  if ((st = A(&n->acc, (size_t)dmax * n->ldT * 4)) || (st = A(&n->work, (size_t)n->work_floats * 4))) {
    hprqp_mlp_destroy(n);
    return st;
  }
  *out = n;
  return HPRQP_OK;
}

static hprqp_status refresh_bf16(hprqp_mlp* n, int l) {
  MlpLayer& y = n->layers[l];
  dim3 grid((unsigned)((y.din + 31) / 32), (unsigned)((y.dout + 31) / 32));
  k_adam_w<<<grid, dim3(32, 8), 0, n->s>>>(y.W, y.mW, y.vW, y.gW, y.dout, y.din, 0, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, y.Wb,
                                            y.ldw, y.WbT, y.ldwt);
  LCU(cudaGetLastError());
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_set_layer(hprqp_mlp* n, int32_t l, const float* W, const float* b) {
  if (!n || l < 0 || l >= n->L) return lfail(HPRQP_INVALID_ARG, "mlp_set_layer: bad layer");
  MlpLayer& y = n->layers[l];
  const size_t nw = (size_t)y.din * y.dout;
  if (W) LCU(cudaMemcpyAsync(y.W, W, nw * 4, cudaMemcpyDefault, n->s));
  if (b) LCU(cudaMemcpyAsync(y.b, b, (size_t)y.dout * 4, cudaMemcpyDefault, n->s));
  LCU(cudaMemsetAsync(y.mW, 0, nw * 4, n->s));
  LCU(cudaMemsetAsync(y.vW, 0, nw * 4, n->s));
  LCU(cudaMemsetAsync(y.mb, 0, (size_t)y.dout * 4, n->s));
  LCU(cudaMemsetAsync(y.vb, 0, (size_t)y.dout * 4, n->s));
  hprqp_status st = refresh_bf16(n, l);
  if (st) return st;
  LCU(cudaStreamSynchronize(n->s));
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_get_layer(hprqp_mlp* n, int32_t l, float* W, float* b) {
  if (!n || l < 0 || l >= n->L) return lfail(HPRQP_INVALID_ARG, "mlp_get_layer: bad layer");
  MlpLayer& y = n->layers[l];
  if (W) LCU(cudaMemcpyAsync(W, y.W, (size_t)y.din * y.dout * 4, cudaMemcpyDefault, n->s));
  if (b) LCU(cudaMemcpyAsync(b, y.b, (size_t)y.dout * 4, cudaMemcpyDefault, n->s));
  LCU(cudaStreamSynchronize(n->s));
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_get_grad(hprqp_mlp* n, int32_t l, float* dW, float* db) {
  if (!n || l < 0 || l >= n->L) return lfail(HPRQP_INVALID_ARG, "mlp_get_grad: bad layer");
  MlpLayer& y = n->layers[l];
  if (dW) LCU(cudaMemcpyAsync(dW, y.gW, (size_t)y.din * y.dout * 4, cudaMemcpyDefault, n->s));
  if (db) LCU(cudaMemcpyAsync(db, y.gb, (size_t)y.dout * 4, cudaMemcpyDefault, n->s));
  LCU(cudaStreamSynchronize(n->s));
  return HPRQP_OK;
}

static hprqp_status mlp_gemm(hprqp_mlp* n, int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda,
                             const uint16_t* B, int64_t ldb, float* C, int64_t ldc) {
  const int sp = pick_splits(M, N, K, n->work_floats, n->sms);
  return gemm(M, N, K, A, lda, B, ldb, C, ldc, sp, n->work, n->s);
}

extern "C" hprqp_status hprqp_mlp_forward(hprqp_mlp* n, const uint16_t* X, int64_t ldx, int32_t batch, float* Y,
                                          int64_t ldy) {
  if (!n || !X || !Y) return lfail(HPRQP_INVALID_ARG, "mlp_forward: null pointer");
  if (batch < 1 || batch > n->maxB) return lfail(HPRQP_INVALID_ARG, "mlp_forward: batch %d not in [1, %d]", batch, n->maxB);
  if (ldx < n->dims[0] || ldx % 8 || ldy < n->dims[n->L]) return lfail(HPRQP_INVALID_ARG, "mlp_forward: bad leading dimension");
  if (!on_device(X) || !on_device(Y)) return lfail(HPRQP_INVALID_ARG, "mlp_forward: X and Y must be device memory");
  hprqp_status st;
  const int B = batch;
  n->B = B;
  {
    const int d0 = n->dims[0];
    dim3 grid((unsigned)((d0 + 31) / 32), (unsigned)((B + 31) / 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, n->s>>>(X, ldx, d0, B, n->actT[0], n->ldT);
    LCU(cudaGetLastError());
  }
  for (int l = 0; l < n->L; ++l) {
    MlpLayer& y = n->layers[l];
    const uint16_t* in = l == 0 ? X : n->actB[l];
    const int64_t ldin = l == 0 ? ldx : round8(y.din);
    if ((st = mlp_gemm(n, y.dout, B, y.din, y.Wb, y.ldw, in, ldin, n->acc, n->ldT))) return st;
    dim3 grid((unsigned)((B + 31) / 32), (unsigned)((y.dout + 31) / 32));
    if (l + 1 < n->L) {
      k_epi<EPI_HIDDEN><<<grid, dim3(32, 8), 0, n->s>>>(n->acc, n->ldT, y.dout, B, y.b, nullptr, nullptr, 0,
                                                          n->actB[l + 1], round8(y.dout), n->actT[l + 1], n->ldT,
                                                          nullptr, 0);
    } else {
      k_epi<EPI_FINAL><<<grid, dim3(32, 8), 0, n->s>>>(n->acc, n->ldT, y.dout, B, y.b, nullptr, nullptr, 0, nullptr, 0,
                                                         nullptr, 0, Y, ldy);
    }
    LCU(cudaGetLastError());
  }
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_backward(hprqp_mlp* n, const float* dY, int64_t lddy) {
  if (!n || !dY) return lfail(HPRQP_INVALID_ARG, "mlp_backward: null pointer");
  if (n->B < 1) return lfail(HPRQP_INVALID_ARG, "mlp_backward: no forward pass yet");
  if (lddy < n->dims[n->L]) return lfail(HPRQP_INVALID_ARG, "mlp_backward: bad leading dimension");
  if (!on_device(dY)) return lfail(HPRQP_INVALID_ARG, "mlp_backward: dY must be device memory");
  hprqp_status st;
  const int B = n->B;
  {
    const int dL = n->dims[n->L];
    dim3 grid((unsigned)((dL + 31) / 32), (unsigned)((B + 31) / 32));
    k_from_batch_f32<<<grid, dim3(32, 8), 0, n->s>>>(dY, lddy, dL, B, n->dzB[n->L - 1], round8(dL), n->dzT[n->L - 1],
                                                     n->ldT);
    LCU(cudaGetLastError());
  }
  for (int l = n->L - 1; l >= 0; --l) {
    MlpLayer& y = n->layers[l];
    // dW = dZ^T X   (dout x din), K = batch
    if ((st = mlp_gemm(n, y.dout, y.din, B, n->dzT[l], n->ldT, n->actT[l], n->ldT, y.gW, y.din))) return st;
    k_rowsum_bf16<<<(int)std::min(y.dout, 65535), 256, 0, n->s>>>(n->dzT[l], n->ldT, y.dout, B, y.gb);
    LCU(cudaGetLastError());
    if (l == 0) break;
    // dX^T = W^T dZ^T  (din x B), masked by the ReLU of the layer below
    if ((st = mlp_gemm(n, y.din, B, y.dout, y.WbT, y.ldwt, n->dzB[l], round8(y.dout), n->acc, n->ldT))) return st;
    dim3 grid((unsigned)((B + 31) / 32), (unsigned)((y.din + 31) / 32));
    k_epi<EPI_MASK><<<grid, dim3(32, 8), 0, n->s>>>(n->acc, n->ldT, y.din, B, nullptr, nullptr, n->actT[l], n->ldT,
                                                      n->dzB[l - 1], round8(y.din), n->dzT[l - 1], n->ldT, nullptr, 0);
    LCU(cudaGetLastError());
  }
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_mlp_adam(hprqp_mlp* n, float lr, float beta1, float beta2, float eps, int64_t t) {
  if (!n || t < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return lfail(HPRQP_INVALID_ARG, "mlp_adam: bad arguments");
  const float bc1 = (float)(1.0 - std::pow((double)beta1, (double)t));
  const float bc2 = (float)(1.0 - std::pow((double)beta2, (double)t));
  for (int l = 0; l < n->L; ++l) {
    MlpLayer& y = n->layers[l];
    dim3 grid((unsigned)((y.din + 31) / 32), (unsigned)((y.dout + 31) / 32));
    k_adam_w<<<grid, dim3(32, 8), 0, n->s>>>(y.W, y.mW, y.vW, y.gW, y.dout, y.din, 1, lr, beta1, beta2, eps, bc1, bc2,
                                              y.Wb, y.ldw, y.WbT, y.ldwt);
    k_adam_b<<<(y.dout + 255) / 256, 256, 0, n->s>>>(y.b, y.mb, y.vb, y.gb, y.dout, lr, beta1, beta2, eps, bc1, bc2);
    LCU(cudaGetLastError());
  }
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ loss, decoder
extern "C" hprqp_status hprqp_ws_loss(const float* O, int64_t ldo, int32_t B, int32_t r, const float* G, const float* R,
                                      int64_t ldr, const double* dd, const float* s, float s_mean, float s_istd,
                                      float alpha, float E, float w_sigma, float* dO, int64_t lddo, int32_t out_cols,
                                      float* loss, void* stream) {
  if (B < 1 || r < 1 || r > 8192 || ldo < 1 + r || lddo < out_cols || out_cols < 1 + r || ldr < B || !(E > 0.f))
    return lfail(HPRQP_INVALID_ARG, "ws_loss: bad sizes");
  if (!O || !G || !R || !dd || !s || !dO || !loss) return lfail(HPRQP_INVALID_ARG, "ws_loss: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  double* part = nullptr;
  LCU(cudaMallocAsync(reinterpret_cast<void**>(&part), (size_t)B * 2 * sizeof(double), st));
  k_ws_loss<<<B, 256, (size_t)r * sizeof(float), st>>>(O, ldo, B, r, G, R, ldr, dd, s, s_mean, s_istd, alpha, E,
                                                       w_sigma, dO, lddo, out_cols, part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_ws_loss_sum<<<1, 32, 0, st>>>(part, B, loss);
    e = cudaGetLastError();
  }
  cudaFreeAsync(part, st);
  if (e != cudaSuccess) return lfail(HPRQP_CUDA_ERROR, "ws_loss: %s", cudaGetErrorString(e));
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_ws_decode(const uint16_t* Phi, int64_t ldphi, int64_t D, int32_t r, const float* O,
                                        int64_t ldo, int32_t B, float alpha, float s_mean, float s_istd,
                                        const double* mu, const double* lo, const double* hi, float* work, double* Z,
                                        int64_t ldz, double* sigma0, void* stream) {
  if (D < 1 || r < 1 || B < 1 || ldo < 1 + r || ldz < D || (B + 31) / 32 > 65535 || (D + 31) / 32 > (int64_t)INT32_MAX)
    return lfail(HPRQP_INVALID_ARG, "ws_decode: bad sizes");
  if (!Phi || !O || !mu || !lo || !hi || !work || !Z) return lfail(HPRQP_INVALID_ARG, "ws_decode: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t ldl = round8(r);
  uint16_t* ell = nullptr;
  LCU(cudaMallocAsync(reinterpret_cast<void**>(&ell), (size_t)B * ldl * 2, st));
  k_cast<float><<<(int)std::min(B, 65535), 256, 0, st>>>(O + 1, B, r, ldo, nullptr, 1.0, ell, ldl, nullptr);
  cudaError_t e = cudaGetLastError();
  hprqp_status s2 = HPRQP_OK;
  if (e == cudaSuccess) s2 = gemm(D, B, r, Phi, ldphi, ell, ldl, work, B, 1, nullptr, st);
  if (e == cudaSuccess && s2 == HPRQP_OK) {
    dim3 grid((unsigned)((D + 31) / 32), (unsigned)((B + 31) / 32));
    k_decode<<<grid, dim3(32, 8), 0, st>>>(work, D, B, alpha, mu, lo, hi, Z, ldz);
    e = cudaGetLastError();
    if (e == cudaSuccess && sigma0) {
      k_sigma0<<<(B + 127) / 128, 128, 0, st>>>(O, ldo, B, s_mean, s_istd, sigma0);
      e = cudaGetLastError();
    }
  }
  cudaFreeAsync(ell, st);
  if (s2) return s2;
  if (e != cudaSuccess) return lfail(HPRQP_CUDA_ERROR, "ws_decode: %s", cudaGetErrorString(e));
  return HPRQP_OK;
}
