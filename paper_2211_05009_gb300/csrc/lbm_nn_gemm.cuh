// lbm_nn_gemm.cuh -- BF16 tensor-core GEMM with FP32 accumulation for the warm-start network.
//
//   C[M][N] (op)= sum_k A[M][K] * B[N][K]      (both operands K-contiguous, "NT" form)
//
// One form serves every convolution product of the network (forward, data gradient, weight
// gradient), with the operands laid out by the im2col kernels.  Block tile 64 x 64, K step 32,
// 4 warps of 32 x 32; operands staged to shared memory with cp.async (16-byte chunks, zero-fill
// outside the matrix), fragments loaded with ldmatrix, products by mma.sync m16n8k16 (BF16 in,
// FP32 accumulate).  Split-K over gridDim.z adds partial products into C atomically.
// Requirements: K, lda, ldb multiples of 8 (16-byte rows); pointers 16-byte aligned.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
namespace nn {

enum GemmOp { kStore = 0, kAccumulate = 1, kAtomicAdd = 2 };

cudaError_t gemm_bf16_nt(int M, int N, int K, const __nv_bfloat16* A, int lda,
                         const __nv_bfloat16* B, int ldb, float* C, int ldc, GemmOp op,
                         int split_k, cudaStream_t st);

// The same product on the 5th-generation tensor cores (tcgen05.mma, TMEM accumulator).
// trans_c stores C[n][m] (element (m, n) at C + n*ldc + m) instead of C[m][n]; split_k > 1
// requires kAtomicAdd.  err: device int set to 1 if a bounded wait ran out (result incomplete).
cudaError_t gemm_bf16_nt_umma(int M, int N, int K, const __nv_bfloat16* A, int lda,
                              const __nv_bfloat16* B, int ldb, float* C, int ldc, GemmOp op, bool trans_c,
                              int split_k, int* err, cudaStream_t st);

// C = conv3x3(x1 ++ x2) as the same product with A = the pixel-major im2col (k = ci*9 + ky*3 + kx,
// padding 1, zeros past (c1 + c2)*9), gathered on the fly from the FP32 [C][H][W] inputs and
// rounded to BF16 exactly as the explicit im2col does (so the result is bitwise that of
// im2col + gemm_bf16_nt_umma).  M = H*W pixels, Wt = [N][K] BF16 weights (K a multiple of 8,
// >= (c1 + c2)*9), N <= 256.
cudaError_t conv3x3_bf16_umma(const float* x1, int c1, const float* x2, int c2, int H, int W, int K,
                              const __nv_bfloat16* Wt, int N, float* C, int ldc, GemmOp op, bool trans_c, int* err,
                              cudaStream_t st);

// The same convolution with the input stored channels-last in BF16 and K ordered tap-major, so
// that each 128 x 64 A tile is one 3-D TMA box (no gather on the SM).  Cp = conv_cp(c1 + c2) (the
// channels rounded up to 64, zero padded).  xs: scratch of H*W*Cp BF16 that receives the
// channels-last input; Wtap: [N][9 * Cp] BF16 from weights_tap_major.  H*W a multiple of 128 and
// W a multiple or a divisor of 128, else cudaErrorInvalidValue (nothing launched).  The sums are
// those of the explicit path in another order, so results agree to FP32 rounding, not bitwise.
int conv_cp(int c);
cudaError_t weights_tap_major(const __nv_bfloat16* Wt, int ldk, int C, int N, __nv_bfloat16* Wtap, cudaStream_t st);
cudaError_t conv3x3_bf16_tma(const float* x1, int c1, const float* x2, int c2, int H, int W, const __nv_bfloat16* Wtap,
                             int N, float* C, int ldc, GemmOp op, bool trans_c, __nv_bfloat16* xs, int* err,
                             cudaStream_t st);

}  // namespace nn
}  // namespace lbm
