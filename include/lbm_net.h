/*
 * lbm_net.h -- the learned warm start (C ABI): a 3D convolutional encoder-decoder that
 * maps the cavity geometry (wall distance, heated-face mask) and log10 Ra, Pr to the
 * steady fields (u, v, w, T), trained on steady states the solver produces, and used to
 * start the solver near its steady state.  The paper has no learned component; this is
 * an accelerator around the method of arXiv:1710.04751, never a replacement: the
 * warm-started solver still runs until its own convergence criterion holds.
 *
 * Arithmetic: BF16 operands on the tcgen05 tensor cores with FP32 accumulation (the
 * forward convolutions, the input gradients and the weight gradients are implicit GEMMs
 * that read their operand tiles straight from the activations and output gradients: no
 * im2col matrix), FP32 master weights and Adam moments.
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

/* 3x3x3 convolution with zero padding as an implicit GEMM on the tensor cores (the
 * network's convolutions, exposed for tests and reuse).  X: device BF16 activations
 * [batch][n][n][n][cin], channels last (voxel ((b n + z) n + y) n + x); W: device BF16
 * weights [cout][ldw] with K index tap * cin + ci, tap = (kz 3 + ky) 3 + kx reading the
 * input at (z + kz - 1, y + ky - 1, x + kx - 1) (ldw >= 27 cin, a multiple of 8); out
 * [batch n^3][cout]: LBM_CONV_BIAS_RELU_BF16 writes BF16 max(y + bias, 0) (bias: device
 * FP32 [cout]), LBM_CONV_F32 writes the FP32 sums y.  Each K block's operand tile is one
 * TMA box of X shifted by the tap, zero-filled outside the grid: no im2col matrix.  cin a
 * multiple of 32, n a power of two in 2..256, cout <= 256, 16-byte aligned bases; else
 * LBM_EINVAL.  Waits for `cuda_stream` (bounded); LBM_ETIMEOUT as lbm_nn_gemm_bf16. */
enum { LBM_CONV_BIAS_RELU_BF16 = 0, LBM_CONV_F32 = 1 };

/* dWT[r][co] += sum over voxels v of X[v + shift(tap)][ci] dZ[v][co], r = tap cin + ci (the
 * weight gradient of lbm_nn_conv3d_bf16's convolution, transposed: [Kp][cout], row stride
 * cout; rows 27 cin .. Kp - 1 receive zeros), as an implicit GEMM that reads both operands
 * in place: every A tile is four TMA boxes of X (32 channels x 64 voxels each, shifted by
 * the tap, zero-filled outside the grid), every B tile boxes of dZ; no im2col matrix and no
 * transpose.  X: device BF16 [batch][n][n][n][cin] as for lbm_nn_conv3d_bf16; dZ: device
 * BF16 [batch n^3][cout], the output gradient.  The voxels are split `splits` ways; the
 * splits' partial tiles go to `ws` (device FP32 scratch of at least splits Kp cout values)
 * and are added to dWT in split order, so the result is the same on every run.  n a power
 * of two in 2..256, cin a multiple of 32, cout a multiple of 8 in 8..256, 16-byte aligned
 * bases; else LBM_EINVAL.  Waits for `cuda_stream` (bounded); LBM_ETIMEOUT as
 * lbm_nn_gemm_bf16. */
int lbm_nn_conv3d_wgrad_bf16(const void* X, int batch, int n, int cin, const void* dZ, int cout, int Kp,
                             float* ws, int64_t ws_floats, int splits, float* dWT, void* cuda_stream);
int lbm_nn_conv3d_bf16(const void* X, int batch, int n, int cin, const void* W, int64_t ldw,
                       int cout, const float* bias, void* out, int mode, void* cuda_stream);

/* Diagnostic of the bounded waits inside the tensor-core kernels (the paper has no
 * counterpart).  Launches the GEMM kernel on one 128 x 32 tile with its operand loads
 * withheld, so that the MMA thread's wait for its first operand stage can only run out
 * (after 10 ms, instead of the 2 s every real launch allows).  The kernel then records
 * the timeout in the device's error word, issues no MMA, frees its tensor memory and
 * returns; the call reads and clears the word.  Returns LBM_ETIMEOUT when that path
 * worked (later GEMMs run normally), LBM_ECUDA otherwise.  Nothing faults or hangs:
 * this is how the timeout path is tested on a shared GPU. */
int lbm_nn_gemm_timeout_probe(void* cuda_stream);

/* ---- the network ------------------------------------------------------------------- */

typedef struct lbm_net lbm_net;

typedef struct {
    int n;            /* grid edge the network is built for: a multiple of 8, 8..256 */
    int max_batch;    /* samples per call at most */
    int c1, c2, c3;   /* channels at the three levels n, n/2, n/4 (multiples of 8;
                         c1 <= 64) */
    uint64_t seed;    /* He-normal initial weights from splitmix64 + Box-Muller */
    float lr, beta1, beta2, eps;  /* Adam (Kingma & Ba 2015) */
    void* cuda_stream;            /* cudaStream_t or NULL */
} lbm_net_config;

/* n 64, max_batch 2, channels 32/64/128 (1.85 M parameters), seed 1, lr 1e-3,
 * betas 0.9 / 0.999, eps 1e-8, NULL stream. */
void lbm_net_default_config(lbm_net_config* cfg);

/* Architecture (a U-Net): conv 4->c1, c1->c1 | avg-pool | c1->c2, c2->c2 | avg-pool |
 * c2->c3, c3->c3, c3->c3 | nearest up, concat | c3+c2->c2, c2->c2 | up, concat |
 * c2+c1->c1, c1->c1 | 1x1 c1->4.  Every conv 3x3x3 with zero padding, bias and ReLU; the
 * 1x1 head is linear.  Inputs per voxel: distance to the nearest wall / n, heated-face
 * mask (+1 on the hot layer, -1 on the cold one), and the sample's two encoded scalars
 * (lbm_net_encode).  Outputs per voxel: u_x, u_y, u_z divided by U0, and 2 T. */
int lbm_net_create(const lbm_net_config* cfg, lbm_net** out);
void lbm_net_destroy(lbm_net* net);
int64_t lbm_net_param_count(const lbm_net* net);

/* The two encoded scalars of a sample: (log10 Ra - 4.5) / 1.5, (log10 Pr - 0.345) / 0.5. */
void lbm_net_encode(double Ra, double Pr, float* out2);

/* Parameters (grads = 0) or the gradients of the last lbm_net_gradients /
 * lbm_net_train_step (grads = 1) to a HOST array of param_count floats: per conv layer
 * W [cout][27 cin] (column (kz*3 + ky)*3 + kx)*cin + ci for the input at
 * (z + kz - 1, y + ky - 1, x + kx - 1)) then b [cout]; then the head W [4][c1], b [4]. */
int lbm_net_get_params(lbm_net* net, float* host, int64_t count, int grads);
int lbm_net_set_params(lbm_net* net, const float* host, int64_t count);

/* Predictions for `batch` samples: scalars = HOST array [batch][2] (lbm_net_encode);
 * out = DEVICE array [batch][n^3][4] FP32, voxel ((b*n + z)*n + y)*n + x. */
int lbm_net_forward(lbm_net* net, int batch, const float* scalars, float* out);
/* Forward and backward without an update: *loss (HOST, may be NULL) = mean squared
 * error against targets (DEVICE, [batch][n^3][4]); gradients via lbm_net_get_params. */
int lbm_net_gradients(lbm_net* net, int batch, const float* scalars, const float* targets,
                      double* loss);
/* The Adam learning rate of the following updates (> 0). */
int lbm_net_set_lr(lbm_net* net, float lr);
/* lbm_net_gradients followed by one Adam update of every parameter.  Every gradient and
 * the loss is summed in a fixed order and every gradient element is written by plain
 * stores (no floating-point atomics anywhere in the network), so the same seed, data and
 * sequence of calls give bitwise identical parameters and losses on every run. */
int lbm_net_train_step(lbm_net* net, int batch, const float* scalars, const float* targets,
                       double* loss);
const char* lbm_net_last_error(const lbm_net* net);

/* Stored tensors of the last lbm_net_forward / lbm_net_gradients / lbm_net_train_step call,
 * for inspection (the per-element checks of the kernels use them).  Activations, voxel-major
 * [sample][voxel][channel] at their level's grid (n, n/2 or n/4): the input features X0,
 * the ReLU outputs A0 S1 | A2 S2 | A4 A5 A6 | A7 A8 | A9 A10 of the eleven convolutions,
 * the pooled P1, P2 and the concatenations C2 = [up(A6), S2], C1 = [up(A8), S1]: BF16
 * (2 bytes each, as stored).  The outputs OUT [sample][n^3][4] and, after a gradient call,
 * the gradients of the loss with respect to OUT and each activation (the D_* ids): FP32.
 * Copies the first `batch` samples (count = batch * voxels * channels elements) into
 * caller-owned host memory, after a bounded wait.  LBM_EINVAL for an unknown id, a batch
 * outside 1..max_batch or a wrong count. */
enum {
    LBM_NET_X0 = 0, LBM_NET_A0, LBM_NET_S1, LBM_NET_P1, LBM_NET_A2, LBM_NET_S2, LBM_NET_P2,
    LBM_NET_A4, LBM_NET_A5, LBM_NET_A6, LBM_NET_C2, LBM_NET_A7, LBM_NET_A8, LBM_NET_C1,
    LBM_NET_A9, LBM_NET_A10, LBM_NET_OUT,
    LBM_NET_D_A10, LBM_NET_D_A9, LBM_NET_D_C1, LBM_NET_D_S1, LBM_NET_D_A8, LBM_NET_D_A7,
    LBM_NET_D_C2, LBM_NET_D_S2, LBM_NET_D_A6, LBM_NET_D_A5, LBM_NET_D_A4, LBM_NET_D_P2,
    LBM_NET_D_A2, LBM_NET_D_P1, LBM_NET_D_A0, LBM_NET_D_OUT, LBM_NET_TENSORS
};
int lbm_net_tensor(lbm_net* net, int which, int batch, void* host, int64_t count);

/* ---- the bridge to the solver ------------------------------------------------------- */

/* Training targets of a context's current state into a DEVICE array [ncell][4] FP32:
 * (u_x, u_y, u_z) / U0 and 2 T, u and T as lbm_fields defines them. */
int lbm_net_targets(lbm_ctx* ctx, float* out);
/* Start a context from a prediction: pred = DEVICE array [m^3][4] on a cell-centred m^3
 * grid covering the cavity, resampled trilinearly onto the context's grid (identity
 * when m equals it), scaled back (u = p U0, T = p / 2), and set as equilibria with
 * rho = 1 followed by `iterations` rounds of the consistent initialisation
 * (lbm_init_fields). */
int lbm_net_warm_start(lbm_ctx* ctx, const float* pred, int m, int iterations);

#ifdef __cplusplus
}
#endif

#endif /* LBM_NET_H */
