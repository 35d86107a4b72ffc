// Arithmetic issue-rate probe (hprqp_fp64_rate): the FP64 roof that bounds the kernels of
// this library on GB300, measured instead of assumed.
//
// Every thread of a full wave of blocks (all resident at once) runs `iters` rounds of eight
// independent dependency chains of one operation, with the first `lanes` lanes of each warp
// active.  Each block records the SM clock (clock64) at its start and end; the span over all
// blocks and the kernel's CUDA-event duration give the SM clock, and the thread operations
// divided by (SMs x cycles) give the rate in lanes per clock per SM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/hprqp.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_rate(int iters, int lanes, double ca, double cb,
                                                        double* sink, long long* span) {
  long long t0 = clock64();
  const int lane = threadIdx.x & 31;
  if (lane < lanes) {
    if (OP <= 2) {
      double a[kChains];
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
      for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) {
          if (OP == 0) a[k] = fma(a[k], ca, cb);
          else if (OP == 1) a[k] = a[k] + cb;
          else a[k] = a[k] * ca;
        }
      }
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < kChains; k++) s += a[k];
      if (s == -1.0) sink[blockIdx.x] = s;   // never true for these inputs; keeps the chains live
    } else {
      float a[kChains];
      const float fa = (float)ca, fb = (float)cb;
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
      for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], fa, fb);
      }
      float s = 0.0f;
#pragma unroll
      for (int k = 0; k < kChains; k++) s += a[k];
      if (s == -1.0f) sink[blockIdx.x] = s;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    span[2 * blockIdx.x] = t0;
    span[2 * blockIdx.x + 1] = t1;
  }
}

template <int OP>
cudaError_t run(int grid, int iters, int lanes, double* sink, long long* span, cudaStream_t s) {
  k_rate<OP><<<grid, kProbeThreads, 0, s>>>(iters, lanes, 0.9999999, 1e-9, sink, span);
  return cudaGetLastError();
}

}  // namespace

extern "C" hprqp_status hprqp_fp64_rate(int32_t op, int32_t lanes, double* lanes_per_clk, double* sm_mhz,
                                        double* ops_per_s) {
  if (op < 0 || op > 3 || lanes < 1 || lanes > 32 || !lanes_per_clk) return HPRQP_INVALID_ARG;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HPRQP_CUDA_ERROR;
  int occ = 0;
  const void* fk = op == 0 ? (const void*)k_rate<0> : op == 1 ? (const void*)k_rate<1> : op == 2 ? (const void*)k_rate<2>
                                                                                               : (const void*)k_rate<3>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk, kProbeThreads, 0) != cudaSuccess || occ < 1) occ = 1;
  const int grid = sms * occ;   // one full wave: every block resident from the start
  // about 20 ms of work at the expected rates (FP64 ~2 lanes/clk/SM, FP32 ~128)
  const int iters = op == 3 ? 65536 : 2048;
  double* sink = nullptr;
  long long* span = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  hprqp_status st = HPRQP_OK;
  if (cudaMalloc(&sink, sizeof(double) * grid) != cudaSuccess || cudaMalloc(&span, sizeof(long long) * 2 * grid) != cudaSuccess) {
    st = HPRQP_OOM;
  }
  if (st == HPRQP_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = HPRQP_CUDA_ERROR;
  float ms = 0.0f;
  long long lo = 0, hi = 0;
  if (st == HPRQP_OK) {
    auto go = [&]() -> cudaError_t {
      switch (op) {
        case 0: return run<0>(grid, iters, lanes, sink, span, 0);
        case 1: return run<1>(grid, iters, lanes, sink, span, 0);
        case 2: return run<2>(grid, iters, lanes, sink, span, 0);
        default: return run<3>(grid, iters, lanes, sink, span, 0);
      }
    };
    cudaError_t e = go();   // warm-up (clocks ramp, code loads)
    if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = go();
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    long long* hs = nullptr;
    if (e == cudaSuccess) {
      hs = new long long[2 * (size_t)grid];
      e = cudaMemcpy(hs, span, sizeof(long long) * 2 * grid, cudaMemcpyDeviceToHost);
    }
    if (e == cudaSuccess) {
      // clock64 counts per SM; blocks of one SM share a counter, so the longest per-SM span
      // is the cycles that SM spent (the counters of different SMs are not aligned)
      long long worst = 0;
      for (int b = 0; b < grid; b++) worst = std::max(worst, hs[2 * b + 1] - hs[2 * b]);
      lo = 0;
      hi = worst;
    }
    delete[] hs;
    if (e != cudaSuccess) st = HPRQP_CUDA_ERROR;
  }
  if (st == HPRQP_OK) {
    const double cycles = (double)(hi - lo);
    const double thread_ops = (double)grid * kProbeThreads / 32.0 * lanes * (double)iters * kChains;
    *lanes_per_clk = cycles > 0 ? thread_ops / ((double)sms * cycles) : 0.0;
    if (sm_mhz) *sm_mhz = ms > 0 ? cycles / (ms * 1e3) : 0.0;
    if (ops_per_s) *ops_per_s = ms > 0 ? thread_ops / (ms * 1e-3) : 0.0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (span) cudaFree(span);
  return st;
}
