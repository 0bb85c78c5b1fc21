/*
 * lbm_net.h -- the learned warm start (C ABI): a 3D convolutional encoder-decoder that
 * maps the cavity geometry (wall distance, heated-face mask) and log10 Ra, Pr to the
 * steady fields (u, v, w, T), trained on steady states the solver produces, and used to
 * start the solver near its steady state.  The paper has no learned component; this is
 * an accelerator around the method of arXiv:1710.04751, never a replacement: the
 * warm-started solver still runs until its own convergence criterion holds.
 *
 * Arithmetic: BF16 operands on the tcgen05 tensor cores with FP32 accumulation (every
 * convolution is a GEMM over an im2col matrix), FP32 master weights and Adam moments.
 *
 * Errors follow include/lbm.h (LBM_OK or a negative LBM_E* code, the message in
 * lbm_last_error(NULL)).  Device pointers are caller-owned.
 */
#ifndef LBM_NET_H
#define LBM_NET_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Output modes of lbm_nn_gemm_bf16. */
enum { LBM_GEMM_F32 = 0, LBM_GEMM_BF16 = 1, LBM_GEMM_F32_ADD = 2 };

/* C[M][N] = sum_k A[m][k] B[n][k] on the tensor cores (building block of the network,
 * exposed for tests and reuse).  A, B: device BF16, row-major, row strides lda, ldb
 * (elements; multiples of 8; 16-byte aligned bases); C: device FP32 (LBM_GEMM_F32,
 * LBM_GEMM_F32_ADD: added atomically, `splits` > 1 splits K across CTAs) or BF16, row
 * stride ldc.  Runs on `cuda_stream` (NULL: legacy stream) and waits for it (bounded).
 * LBM_EINVAL for bad shapes or alignment; LBM_ETIMEOUT if a wait inside the kernel ran
 * out (the kernel then stores nothing). */
int lbm_nn_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                     int64_t ldc, int M, int N, int K, int out_mode, int splits,
                     void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NET_H */
