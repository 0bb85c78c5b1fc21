// nn.h -- declarations shared by the translation units of the warm-start network
// (tensor-core GEMM, layer kernels, the network itself).  Not installed.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
namespace nn {

enum { GEMM_F32 = 0, GEMM_BF16 = 1, GEMM_F32_ATOMIC = 2 };

// C[M][N] (row stride ldc) = (or +=, GEMM_F32_ATOMIC) sum_k A[m][k] B[n][k]; A and B BF16
// row-major with row strides lda, ldb (elements, multiples of 8, 16-byte aligned bases);
// FP32 accumulation on the tensor cores; `splits` > 1 splits K (atomic mode only).  A
// timeout inside the kernel writes a non-zero code to *err (device memory).
cudaError_t gemm_bf16(const __nv_bfloat16* A, long long lda, const __nv_bfloat16* B,
                      long long ldb, void* C, long long ldc, int M, int N, int K, int out_mode,
                      int splits, int* err, cudaStream_t st);

}  // namespace nn
}  // namespace lbm
