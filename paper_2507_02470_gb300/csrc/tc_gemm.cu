// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05) of sm_103a.
//
// One CTA of 128 threads computes a 128 x BN tile of C = A B^T:
//   - warp 0 / lane 0 streams 128 x 64 tiles of A and BN x 64 tiles of B into a ring of
//     kStages shared-memory stages with the tensor-memory-access engine (TMA, 128-byte
//     swizzle, zero fill past the tensor edges), each stage guarded by a "full" mbarrier
//     that counts the bytes in flight;
//   - warp 1 / lane 0 issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction, four per
//     stage) into an FP32 accumulator in tensor memory (TMEM), and releases each stage with
//     tcgen05.commit on its "empty" mbarrier once the MMAs that read it have finished;
//   - after the last stage a commit on the "done" mbarrier hands the accumulator to all four
//     warps, which read it back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31, i.e.
//     rows 32w.. of the tile) and store FP32 rows to global memory.
// Every mbarrier wait is bounded: when a wait gives up the kernel records an error code in
// g_tc_error, stops issuing work, still commits the done barrier so the other warps are not
// left waiting, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "tc_gemm.cuh"

namespace hprqp {
namespace tc {
namespace {

constexpr int kBM = 128;                       // tile rows = TMEM lanes
constexpr int kBK = 64;                        // K per stage: one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr uint32_t kATile = kBM * kBK * 2;     // bytes of one A stage
constexpr uint32_t kSpin = 1u << 22;           // polls of one bounded wait (about a second)

__device__ int g_tc_error;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// non-blocking test of the phase with the given parity
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int code) {
  for (uint32_t i = 0; i < kSpin; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (i >= 64) __nanosleep(200);
  }
  atomicCAS(&g_tc_error, 0, code);
  return false;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile stored as 128-byte rows with the
// 128-byte swizzle (the layout the TMA writes): start address >> 4 in bits 0-13, leading
// byte offset 16 B (unused for swizzled K-major tiles) in bits 16-29, stride byte offset
// 1024 B (eight rows) in bits 32-45, the fixed version field 1 in bits 46-48, base offset 0
// (stages are 1024-byte aligned), swizzle mode 2 (128-byte) in bits 61-63.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// BF16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive FP32 columns of the calling thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int BN>
constexpr uint32_t smem_bytes() {
  return 1024 + kStages * (kATile + (uint32_t)BN * kBK * 2);
}

template <int BN>
__global__ void __launch_bounds__(128, 1)
    k_gemm_bf16(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, float* __restrict__ C,
                int64_t ldc, int64_t split_stride, int M, int N, int kb_total, int kb_per, int vec) {
  static_assert(BN == 64 || BN == 128 || BN == 256, "TMEM columns must be a power of two >= 32");
  constexpr uint32_t kBTile = (uint32_t)BN * kBK * 2;
  __shared__ __align__(8) uint64_t bar_full[kStages];
  __shared__ __align__(8) uint64_t bar_empty[kStages];
  __shared__ __align__(8) uint64_t bar_done;
  __shared__ uint32_t tmem_slot;
  extern __shared__ uint8_t dsm[];
  const uint32_t base = (smem_u32(dsm) + 1023u) & ~1023u;   // stages start on 1024-byte boundaries

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int kb0 = blockIdx.z * kb_per;
  const int nkb = min(kb0 + kb_per, kb_total) - kb0;        // >= 1 (host)

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&bar_full[s]), 1);
      mbar_init(smem_u32(&bar_empty[s]), 1);
    }
    mbar_init(smem_u32(&bar_done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: stage s of round r waits for the MMAs of round r-1 to release it
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(smem_u32(&bar_empty[s]), ph ^ 1u, 1)) break;
      const uint32_t fb = smem_u32(&bar_full[s]);
      mbar_expect_tx(fb, kATile + kBTile);
      const int kx = (kb0 + i) * kBK;   // multiple of 64 elements: 16-byte aligned
      tma_load_2d(base + s * kATile, &ta, fb, kx, m0);
      tma_load_2d(base + kStages * kATile + s * kBTile, &tb, fb, kx, n0);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      const uint32_t ph = (uint32_t)(i / kStages) & 1u;
      if (!mbar_wait(smem_u32(&bar_full[s]), ph, 2)) break;
      tc_fence_after();
      const uint64_t ad = sdesc_sw128(base + s * kATile);
      const uint64_t bd = sdesc_sw128(base + kStages * kATile + s * kBTile);
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk)   // +32 bytes along K inside the swizzle row
        mma_bf16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(smem_u32(&bar_empty[s]));
    }
    mma_commit(smem_u32(&bar_done));    // arrives when every MMA issued above has completed
  }
  __syncwarp();

  // epilogue: TMEM lane (32 warp + lane) holds row m0 + 32 warp + lane of the tile
  const bool ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&bar_done), 0, 3));
  tc_fence_after();
  if (ok) {
    const int row = m0 + warp * 32 + lane;
    float* crow = C + (int64_t)blockIdx.z * split_stride + (int64_t)row * ldc;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
      const int col = n0 + c0;
      if (row < M && col < N) {
        if (vec && col + 32 <= N) {
          float4* d = reinterpret_cast<float4*>(crow + col);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            d[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                               __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col + j < N) crow[col + j] = __uint_as_float(r[j]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
  }
}

// C[i][j] = sum_s work[s][i][j], s = 0..S-1 in order
__global__ void k_splitk_sum(const float* __restrict__ work, int S, int64_t M, int64_t N, float* __restrict__ C,
                             int64_t ldc) {
  const int64_t total = M * N, stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += stride) {
    float acc = 0.f;
    for (int s = 0; s < S; ++s) acc += work[(int64_t)s * total + e];
    C[(e / N) * ldc + (e % N)] = acc;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder(cudaError_t* err) {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static cudaError_t e0 = cudaSuccess;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    e0 = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e0 == cudaSuccess && q != cudaDriverEntryPointSuccess) e0 = cudaErrorSymbolNotFound;
    if (e0 == cudaSuccess) fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  *err = e0;
  return fn;
}

// 2-D map over a rows x cols BF16 matrix with leading dimension ld; boxes of 64 x box_rows
cudaError_t make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  cudaError_t e;
  auto fn = encoder(&e);
  if (!fn) return e;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
cudaError_t launch(const CUtensorMap& ta, const CUtensorMap& tb, float* C, int64_t ldc, int64_t split_stride,
                   int64_t M, int64_t N, int kb_total, int kb_per, int splits, int vec, cudaStream_t s) {
  constexpr uint32_t bytes = smem_bytes<BN>();
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  });
  if (attr != cudaSuccess) return attr;
  dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + BN - 1) / BN), (unsigned)splits);
  k_gemm_bf16<BN><<<grid, 128, bytes, s>>>(ta, tb, C, ldc, split_stride, (int)M, (int)N, kb_total, kb_per, vec);
  return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                      float* C, int64_t ldc, int splits, float* work, cudaStream_t stream, const char** why) {
  auto bad = [why](const char* w) {
    if (why) *why = w;
    return cudaErrorInvalidValue;
  };
  if (M < 0 || N < 0 || K < 0) return bad("negative size");
  if (M == 0 || N == 0) return cudaSuccess;
  if (M >= (1ll << 31) || N > 65535ll * 64 || K >= (1ll << 31)) return bad("size out of range");
  if (!C || ldc < N) return bad("C is null or ldc < N");
  if (K == 0) {
    for (int64_t i = 0; i < M; ++i) {   // rows may be strided: one memset per row
      cudaError_t e = cudaMemsetAsync(C + i * ldc, 0, (size_t)N * sizeof(float), stream);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!A || !B) return bad("A or B is null");
  if (lda < K || ldb < K) return bad("lda and ldb must be >= K");
  if (lda % 8 || ldb % 8) return bad("lda and ldb must be multiples of 8 (16-byte rows)");
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return bad("A and B must be 16-byte aligned");
  const int kb_total = (int)((K + kBK - 1) / kBK);
  splits = std::max(1, std::min(splits, kb_total));
  const int kb_per = (kb_total + splits - 1) / splits;
  splits = (kb_total + kb_per - 1) / kb_per;   // no empty split
  if (splits > 1 && !work) return bad("splits > 1 needs a work buffer of splits*M*N floats");
  if (splits > 65535) return bad("too many splits");
  // tile width: 256 columns (128 x 256 accumulator, 256 TMEM columns) when N is wide enough
  // to keep many tiles, else 128 or 64
  const int BN = N <= 64 ? 64 : N < 512 ? 128 : 256;
  CUtensorMap ta, tb;
  cudaError_t e;
  if ((e = make_map(&ta, A, M, K, lda, kBM)) != cudaSuccess) return e;
  if ((e = make_map(&tb, B, N, K, ldb, BN)) != cudaSuccess) return e;
  float* out = splits > 1 ? work : C;
  const int64_t ld = splits > 1 ? N : ldc;
  const int vec = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && ld % 4 == 0) ? 1 : 0;
  e = BN == 64    ? launch<64>(ta, tb, out, ld, M * N, M, N, kb_total, kb_per, splits, vec, stream)
      : BN == 128 ? launch<128>(ta, tb, out, ld, M * N, M, N, kb_total, kb_per, splits, vec, stream)
                  : launch<256>(ta, tb, out, ld, M * N, M, N, kb_total, kb_per, splits, vec, stream);
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t total = M * N;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  k_splitk_sum<<<blocks, 256, 0, stream>>>(work, splits, M, N, C, ldc);
  return cudaGetLastError();
}

int gemm_error_flag() {
  int v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (v) cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  return v;
}

}  // namespace tc
}  // namespace hprqp
