// nn.h -- declarations shared by the translation units of the warm-start network
// (tensor-core GEMM, layer kernels, the network itself).  Not installed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
namespace nn {

enum { GEMM_F32 = 0, GEMM_BF16 = 1, GEMM_F32_ATOMIC = 2, GEMM_F32_SPLITS = 3 };

// C[M][N] (row stride ldc) = (or +=, GEMM_F32_ATOMIC) sum_k A[m][k] B[n][k]; A and B BF16
// row-major with row strides lda, ldb (elements, multiples of 8, 16-byte aligned bases);
// FP32 accumulation on the tensor cores; `splits` > 1 splits K (GEMM_F32_ATOMIC, or
// GEMM_F32_SPLITS: split z writes its partial result to C + z * M * ldc).  A timeout
// inside the kernel writes a non-zero code to *err (device memory).
cudaError_t gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
                      long long ldb, void* C, long long ldc, int M, int N, int K, int out_mode,
                      int splits, int* err, cudaStream_t st);

// C += A B^T (FP32 C) with K split across CTAs and the partial results added in split
// order from the workspace ws (gemm_splitk_floats floats): run-to-run identical sums.
cudaError_t gemm_bf16_add_splitk(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
                                 long long ldb, float* C, long long ldc, int M, int N, int K,
                                 int splits, float* ws, size_t ws_floats, int* err, cudaStream_t st);
size_t gemm_splitk_floats(int M, long long ldc, int K, int splits);

// 3x3x3 convolution with zero padding as an implicit GEMM (conv.cu): X [B][n][n][n][cin]
// BF16 channels last, W [cout][ldw] BF16 (K index tap * cin + ci), out [B n^3][cout]:
// CONV_BIAS_RELU_BF16 writes bf16(max(y + bias, 0)), CONV_F32 writes y.  Needs
// conv_implicit_supported (cin a multiple of 32, n a power of two); 16-byte aligned bases.
enum { CONV_BIAS_RELU_BF16 = 0, CONV_F32 = 1 };
bool conv_implicit_supported(int n, int cin, int cout);
cudaError_t conv_implicit(const __nv_bfloat16* X, int B, int n, int cin, const __nv_bfloat16* W,
                          long long ldw, int cout, const float* bias, void* out, int mode, int* err,
                          cudaStream_t st);

// Diagnostic: the GEMM kernel on one tile with its operand loads withheld, so that its
// bounded wait runs out (10 ms) and it records a timeout in *err (see gemm.cu).
cudaError_t gemm_timeout_probe(const __nv_bfloat16* operand, float* C, int* err, cudaStream_t st);

}  // namespace nn
}  // namespace lbm

namespace lbm {
namespace nn {

// layers.cu (channels-last activations, see there)
cudaError_t im2col(const __nv_bfloat16* X, int B, int n, int cin, int Kp, __nv_bfloat16* Xcol,
                   cudaStream_t st);
// XcolT [Kp][M] = im2col(X) transposed (M = B n^3 voxels, row stride M), without the
// intermediate matrix; n a power of two, cin a multiple of 32, M of 8; padding rows zeroed.
bool im2colT_supported(int n, int cin, int64_t M);
cudaError_t im2colT(const __nv_bfloat16* X, int B, int n, int cin, int Kp, __nv_bfloat16* XcolT,
                    cudaStream_t st);
// dWT [Kp][cout] += the weight gradient of a 3x3x3 convolution of X [B n^3][cin] with output
// gradient dZ [B n^3][cout], as an implicit GEMM on both in place (conv.cu): n a power of two
// in 2..256, cin a multiple of 32, cout a multiple of 8 up to 256; ws holds splits Kp cout
// floats (the split partials, added to dWT in split order; accumulate == 0: dWT = the sum).
bool conv_wgrad_implicit_supported(int B, int n, int cin, int cout);
cudaError_t conv_wgrad_implicit(const __nv_bfloat16* X, int B, int n, int cin, const __nv_bfloat16* dZ, int cout,
                                int Kp, float* ws, size_t ws_floats, int splits, float* dWT, int accumulate,
                                int* err, cudaStream_t st);
// C[r][c] = (accumulate ? C[r][c] : 0) + ws[0][r][c] + ws[1][r][c] + ... in split order
// (slices of M ldc floats).
cudaError_t add_splits(const float* ws, int splits, int M, int N, long long ldc, float* C, int accumulate,
                       cudaStream_t st);
cudaError_t transpose(const __nv_bfloat16* in, int64_t R, int64_t C, int64_t ld_in,
                      __nv_bfloat16* out, int64_t ld_out, cudaStream_t st);
cudaError_t bias_relu(const float* Y, const float* bias, int64_t M, int C, __nv_bfloat16* A,
                      int64_t ldA, int c_off, cudaStream_t st);
// Gradient reductions over rows (relu_bwd's db, head_bwd's dW and db, mse's loss) store
// the sum of per-block partial sums, taken in a fixed order: `part` holds kMaxPartialBlocks * C floats
// (relu_bwd), kMaxPartialBlocks * (4 C + 4) floats (head_bwd) or kMaxPartialBlocks
// doubles (mse).
constexpr int kMaxPartialBlocks = 1024;
cudaError_t relu_bwd(const float* dA, const __nv_bfloat16* A, int64_t ldA, int a_off, int64_t M,
                     int C, __nv_bfloat16* dZ, float* db, float* part, cudaStream_t st);
cudaError_t avgpool(const __nv_bfloat16* X, int B, int n, int C, __nv_bfloat16* P, cudaStream_t st);
cudaError_t avgpool_bwd(const float* dP, int B, int n, int C, float* dX, int accumulate,
                        cudaStream_t st);
cudaError_t upsample(const __nv_bfloat16* X, int B, int n, int C, __nv_bfloat16* U, int64_t ldU,
                     int c_off, cudaStream_t st);
cudaError_t upsample_bwd(const float* dU, int64_t ldU, int c_off, int B, int n, int C, float* dX,
                         cudaStream_t st);
cudaError_t copy_channels(const __nv_bfloat16* S, int64_t M, int C, __nv_bfloat16* D, int64_t ldD,
                          int c_off, cudaStream_t st);
cudaError_t slice_grad(const float* dD, int64_t ldD, int c_off, int64_t M, int C, float* dS,
                       int accumulate, cudaStream_t st);
cudaError_t head_fwd(const __nv_bfloat16* A, int64_t M, int C, const float* W, const float* b,
                     float* out, cudaStream_t st);
cudaError_t head_bwd(const float* dOut, const __nv_bfloat16* A, int64_t M, int C, const float* W,
                     float* dA, float* dW, float* db, float* part, cudaStream_t st);
cudaError_t mse(const float* out, const float* target, int64_t count, float* dOut, double* loss,
                double* part, cudaStream_t st);
// Tables of tensors for the one-launch Adam step, weight packing and gradient unpacking.
constexpr int kMaxSegs = 32;
struct AdamSeg {
    float* p;
    const float* g;
    float *m, *v;
    int64_t n;
};
struct AdamTable {
    AdamSeg seg[kMaxSegs];
    int count;
};
// Weights [cout][27 cin] for an input stored with cs >= cin channels: K index tap * cs + ci
// (Wb [cout][Kp]); Wf [cin][Kpf] the mirrored input-gradient weights, or NULL.
struct PackSeg {
    const float* W;
    int cin, cs, cout, Kp, Kpf;
    __nv_bfloat16 *Wb, *Wf;
};
struct PackTable {
    PackSeg seg[kMaxSegs];
    int count;
};
struct UnpackSeg {
    const float* dWT;
    int cout, cin, cs;
    float* gW;
};
struct UnpackTable {
    UnpackSeg seg[kMaxSegs];
    int count;
};
// The tables travel as kernel parameters (__grid_constant__): within the classic 4 KB.
static_assert(sizeof(AdamTable) + 6 * sizeof(float) <= 4096, "Adam table exceeds the parameter space");
static_assert(sizeof(PackTable) <= 4096 && sizeof(UnpackTable) <= 4096, "table exceeds the parameter space");
cudaError_t adam(const AdamTable& t, float lr, float b1, float b2, float eps, int step, cudaStream_t st);
cudaError_t pack_weights(const PackTable& t, cudaStream_t st);
cudaError_t unpack_grad(const UnpackTable& t, cudaStream_t st);
// The 4 input channels in rows of ldx (a multiple of 8; channels 4 .. ldx - 1 written zero).
cudaError_t features(int B, int n, const float* scalars, __nv_bfloat16* X, int ldx, cudaStream_t st);

}  // namespace nn
}  // namespace lbm
