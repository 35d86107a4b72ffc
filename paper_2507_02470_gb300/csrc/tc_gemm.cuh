// BF16 tensor-core GEMM for the learned warm start: C = A * B^T with A (M x K) and B (N x K)
// both row-major with K contiguous ("K-major"), BF16 inputs, FP32 accumulation in tensor
// memory, FP32 output.  Every product of the warm-start network (forward and backward), the
// feature projection and the decoder is written in this one form by choosing which stored
// layout (batch-major or feature-major) plays A and which plays B.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hprqp {
namespace tc {

// Launches C = A B^T (split along K into `splits` parts summed in a fixed order when
// splits > 1, using `work` of splits * M * N floats).  A: M x K with leading dimension lda
// (elements), B: N x K with ldb, C: M x N with ldc.  Requirements checked here: lda, ldb
// multiples of 8 (16-byte rows), A and B 16-byte aligned, lda >= K, ldb >= K, ldc >= N.
// Rows and columns past M, N, K are read as zeros by the copy engine and never written.
// Returns cudaSuccess or the first failing runtime/driver call as a cudaError_t;
// cudaErrorInvalidValue for bad arguments (message in *why when why != nullptr).
cudaError_t gemm_bf16(int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, const void* B, int64_t ldb,
                      float* C, int64_t ldc, int splits, float* work, cudaStream_t stream, const char** why);

// Reads and clears the device flag that a GEMM kernel sets when one of its bounded waits
// gave up (0: none; 1 producer, 2 MMA issuer, 3 epilogue).  Synchronises the device.
int gemm_error_flag();

}  // namespace tc
}  // namespace hprqp
