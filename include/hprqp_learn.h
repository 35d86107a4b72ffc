/* hprqp_learn.h — C ABI of the learned warm start for parametric HPR-QP families.
 *
 * Algorithm 4 may start from any point u^{0,0}: the Halpern step averages every iterate with
 * the starting point of its restart cycle (Step 5 of Algorithm 1, Sec. 2.1, and its use in
 * Algorithm 4), and the paper itself always starts at the origin (Sec. 4.1).  For a family
 * of problems that share A, Q and C and differ in c and the row bounds, this part of the
 * library predicts a starting point (x^0, y^0) and an initial penalty sigma0 from the problem
 * data, with a small multilayer perceptron trained on solutions that hprqp_solve produced
 * for other members of the family.  The prediction only sets the starting point;
 * hprqp_solve still runs to its own stopping test, so a poor prediction costs iterations,
 * never accuracy.
 *
 * The pipeline, all on the GPU:
 *   features  f = P [c; u]               P: d0 x D random projection, D = n + m (GEMM)
 *   network   o = MLP(standardised f)    ReLU hidden layers, BF16 weights and activations,
 *                                        FP32 accumulation on the tensor cores (GEMMs)
 *   decoder   log sigma0 = s_mean + o_0 / s_istd,   ell = alpha o_{1..r},
 *             z0 = clip(mu + Phi ell, lo, hi)    Phi: D x r fixed random basis (GEMM),
 *                                                mu: mean training solution, z0 = (x0, y0)
 *
 * Conventions: BF16 arrays are uint16_t bit patterns; every array argument of the entry
 * points below is DEVICE memory of the current CUDA device unless it says "host"; row-major
 * storage with the stated leading dimension (ld, in elements).  `stream` is a cudaStream_t
 * (NULL: legacy default stream); calls are asynchronous on it unless stated otherwise.
 * Statuses are those of hprqp.h; on failure hprqp_learn_last_error() returns a message.
 */
#ifndef HPRQP_LEARN_H
#define HPRQP_LEARN_H

#include <stdint.h>

#include "hprqp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- tensor-core GEMM
 * C = A B^T with A (M x K, lda) and B (N x K, ldb) BF16, both with K contiguous, and C
 * (M x N, ldc) FP32, computed with tcgen05.mma (FP32 accumulation in tensor memory).
 * splits > 1 splits K into that many parts computed by separate CTAs and summed in a fixed
 * order (deterministic); work must then hold splits * M * N floats.  Entries of A, B past
 * M, N, K are never read.  Requirements: lda, ldb multiples of 8 and >= K; A and B 16-byte
 * aligned; ldc >= N.  Returns HPRQP_INVALID_ARG when they fail, HPRQP_CUDA_ERROR on a
 * launch failure.  Tiles are 128 x BN with BN = 64 (N <= 64), 128 (N < 512) or 256. */
hprqp_status hprqp_gemm_bf16(int64_t M, int64_t N, int64_t K, const uint16_t* A, int64_t lda, const uint16_t* B,
                             int64_t ldb, float* C, int64_t ldc, int32_t splits, float* work, void* stream);

/* Synchronises the device and returns HPRQP_TIMEOUT if a GEMM kernel gave up one of its
 * bounded waits since the last call (the flag is then cleared), HPRQP_OK otherwise. */
hprqp_status hprqp_learn_check(void);

/* ---------------------------------------------------------------- conversions
 * out[i][j] = bf16(((double)x[i][j] - sub[j]) * scale) for j < cols, out[i][j] = 0 for
 * cols <= j < ldo (ldo >= cols); sub may be NULL (zeros).  When rownorm2 is not NULL,
 * rownorm2[i] = sum_j (((double)x[i][j] - sub[j]) * scale)^2 in FP64 (before rounding).
 * Rounding: FP64 -> FP32 -> BF16, each to nearest even; non-finite inputs become 0. */
hprqp_status hprqp_cast_bf16_f64(const double* x, int64_t rows, int64_t cols, int64_t ldx, const double* sub,
                                 double scale, uint16_t* out, int64_t ldo, double* rownorm2, void* stream);
hprqp_status hprqp_cast_bf16_f32(const float* x, int64_t rows, int64_t cols, int64_t ldx, const double* sub,
                                 double scale, uint16_t* out, int64_t ldo, double* rownorm2, void* stream);

/* Mean and inverse standard deviation of each row of F (rows x cols, ld):
 * mean[i] = sum_j F[i][j] / cols, istd[i] = 1 / sqrt(max(var_i, floor)) with the population
 * variance var_i, accumulated in FP64 in a fixed order.  Results FP32. */
hprqp_status hprqp_row_stats(const float* F, int64_t rows, int64_t cols, int64_t ld, float floor, float* mean,
                             float* istd, void* stream);

/* Column means of Z (rows x cols, ld), FP64: mu[j] = sum_i Z[i][j] / rows (fixed order). */
hprqp_status hprqp_col_mean_f64(const double* Z, int64_t rows, int64_t cols, int64_t ld, double* mu, void* stream);

/* Standardised features from the feature-major GEMM output F (d x B, ldf):
 * X[b][j] = bf16((F[j][b] - mean[j]) * istd[j]) batch-major (B x d, ldx >= d; padding 0). */
hprqp_status hprqp_ws_standardize(const float* F, int64_t d, int64_t B, int64_t ldf, const float* mean,
                                  const float* istd, uint16_t* X, int64_t ldx, void* stream);

/* ---------------------------------------------------------------- multilayer perceptron
 * Layer l (0 <= l < nlayers) maps dims[l] -> dims[l+1]: y = W_l x + b_l, followed by ReLU on
 * every layer but the last.  FP32 master weights with BF16 copies W_l and W_l^T used by the
 * GEMMs; activations are stored in BF16 in both batch-major and feature-major layouts; the
 * output of the last layer is FP32.  Gradients are FP32 (dW from GEMMs of BF16 operands).
 * Training uses Adam (Kingma and Ba, 2015) on the master weights. */
typedef struct hprqp_mlp hprqp_mlp;

/* dims: host array of nlayers + 1 widths (each >= 1); max_batch >= 1.  Weights start at 0. */
hprqp_status hprqp_mlp_create(hprqp_mlp** net, int32_t nlayers, const int32_t* dims, int32_t max_batch,
                              void* stream);
/* Copies W (dims[l+1] x dims[l], row-major) and b (dims[l+1]) in FP32, host or device, into
 * layer l and clears its Adam moments. */
hprqp_status hprqp_mlp_set_layer(hprqp_mlp* net, int32_t l, const float* W, const float* b);
/* Copies the FP32 master weights of layer l out (host or device; either may be NULL). */
hprqp_status hprqp_mlp_get_layer(hprqp_mlp* net, int32_t l, float* W, float* b);
/* Y = MLP(X) for X batch-major BF16 (batch x dims[0], ldx >= dims[0], multiple of 8) and Y
 * batch-major FP32 (batch x dims[nlayers], ldy).  1 <= batch <= max_batch.  Keeps the
 * activations for hprqp_mlp_backward. */
hprqp_status hprqp_mlp_forward(hprqp_mlp* net, const uint16_t* X, int64_t ldx, int32_t batch, float* Y, int64_t ldy);
/* Gradients of a loss with dL/dY = dY (batch x dims[nlayers], lddy; FP32; rounded to BF16
 * before the backward GEMMs) with respect to every W_l and b_l, for the batch of the last
 * forward; overwrites the stored gradients. */
hprqp_status hprqp_mlp_backward(hprqp_mlp* net, const float* dY, int64_t lddy);
/* Copies the FP32 gradients of layer l out (host or device; either may be NULL). */
hprqp_status hprqp_mlp_get_grad(hprqp_mlp* net, int32_t l, float* dW, float* db);
/* One Adam step, t >= 1 the step count (bias corrections 1 - beta^t):
 * m = beta1 m + (1-beta1) g;  v = beta2 v + (1-beta2) g^2;
 * W -= lr (m / (1-beta1^t)) / (sqrt(v / (1-beta2^t)) + eps);  BF16 copies refreshed. */
hprqp_status hprqp_mlp_adam(hprqp_mlp* net, float lr, float beta1, float beta2, float eps, int64_t t);
hprqp_status hprqp_mlp_destroy(hprqp_mlp* net);

/* ---------------------------------------------------------------- warm-start loss and decoder
 * Loss of the network output O (B x ldo, FP32; column 0 the standardised log sigma0, columns
 * 1..r the latent o_ell) for one batch, with ell = alpha o_ell and the standardised target
 * s_hat[b] = (s[b] - s_mean) * s_istd of the log sigma targets s:
 *   L = (1/B) sum_b [ w_sigma/2 (O[b][0] - s_hat[b])^2
 *                     + 1/(2E) (alpha^2 o_ell^T G o_ell - 2 alpha o_ell^T R[:,b] + dd[b]) ]
 * which is (1/B) sum_b [ w_sigma/2 (O[b][0]-s_hat[b])^2 + ||mu + Phi ell - z*_b||^2 / (2E) ]
 * for G = Phi^T Phi (r x r, FP32), R = Phi^T (Z* - mu)^T (r x B feature-major, ldr) and
 * dd[b] = ||z*_b - mu||^2.  Writes dO = dL/dO (B x lddo, FP32; columns 1+r..out_cols-1 set
 * to 0) and loss[0] = sigma part, loss[1] = latent part (FP32, summed in a fixed order). */
hprqp_status hprqp_ws_loss(const float* O, int64_t ldo, int32_t B, int32_t r, const float* G, const float* R,
                           int64_t ldr, const double* dd, const float* s, float s_mean, float s_istd, float alpha,
                           float E, float w_sigma, float* dO, int64_t lddo, int32_t out_cols, float* loss,
                           void* stream);

/* Decoder of the network output O (B x ldo, FP32):
 *   ell[b] = bf16(O[b][1..r]),  sigma0[b] = exp(s_mean + O[b][0] / s_istd),
 *   Z[b][i] = clip(mu[i] + alpha sum_k Phi[i][k] ell[b][k], lo[i], hi[i])   (FP64, i < D)
 * with Phi (D x r, ldphi, BF16).  work: D * B floats.  sigma0 may be NULL. */
hprqp_status hprqp_ws_decode(const uint16_t* Phi, int64_t ldphi, int64_t D, int32_t r, const float* O, int64_t ldo,
                             int32_t B, float alpha, float s_mean, float s_istd, const double* mu, const double* lo,
                             const double* hi, float* work, double* Z, int64_t ldz, double* sigma0, void* stream);

/* Message of the last failed call of this header on the calling thread. */
const char* hprqp_learn_last_error(void);

/* ---------------------------------------------------------------- parametric data
 * Replaces c (n), the row bounds l and u (m) of a created problem; A, Q, C and phi are kept.
 * Any pointer may be NULL (unchanged).  Host or device pointers.  Same validation as
 * hprqp_create.  The warm start, if any, is kept. */
hprqp_status hprqp_set_data(hprqp_handle* h, const double* c, const double* l, const double* u);
/* Fixes lambda_A and lambda_Q for later solves (> 0; 0 restores the power method). */
hprqp_status hprqp_set_lambda(hprqp_handle* h, double lambda_A, double lambda_Q);

#ifdef __cplusplus
}
#endif
#endif
