// net.cu -- the warm-start network: a 3D convolutional encoder-decoder (U-Net) on an
// n^3 grid (n a multiple of 8), channels c1, c2, c3 at the levels n, n/2, n/4:
//
//   L0  conv 4 -> c1, L1 conv c1 -> c1                      (level 0)  -> S1
//   pool; L2 conv c1 -> c2, L3 conv c2 -> c2                 (level 1)  -> S2
//   pool; L4 conv c2 -> c3, L5, L6 conv c3 -> c3             (level 2)
//   up, concat S2; L7 conv c3+c2 -> c2, L8 conv c2 -> c2      (level 1)
//   up, concat S1; L9 conv c2+c1 -> c1, L10 conv c1 -> c1     (level 0)
//   head: 1x1 conv c1 -> 4 (linear)
//
// every conv 3x3x3 with zero padding, bias and ReLU; pool = 2x average, up = 2x nearest.
// Inputs: 4 channels (wall distance, heated-face mask, normalised log10 Ra and log10 Pr);
// outputs: (u_x, u_y, u_z) / U0 and 2 T.  Each convolution is a tensor-core GEMM over
// im2col(X), taken implicitly (conv.cu: the operand tiles are TMA boxes of the activations,
// no im2col matrix): forward Y = Xcol W^T; weight gradient dW^T = Xcol^T dZ, split over the
// voxels; input gradient dX = im2col(dZ) Wf^T, the convolution of the output gradient with
// the mirrored, channel-exchanged weights Wf.  Shapes the implicit kernels do not take fall
// back to an explicit im2col matrix and the GEMM of gemm.cu.  FP32 master weights, Adam,
// BF16 operand copies.
#include <math.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../context.h"
#include "lbm_net.h"
#include "nn.h"

using namespace lbm;
using namespace lbm::nn;

namespace {

constexpr int kLayers = 11;
// The 4 input channels are stored in rows of 32 (the rest zero), so that the first
// convolution reads its input like every other layer: implicit GEMMs with 32-channel boxes.
constexpr int kX0 = 32;
static_assert(2 * kLayers + 2 <= kMaxSegs, "one Adam table holds every parameter tensor");

struct Conv {
    int cin, cout, level, K27, Kp, Kpf;  // Kpf: padded 27 cout (input-gradient GEMM)
    int cs;                              // channels of the stored input (cin, kX0 for layer 0)
    float *W, *b, *gW, *gb, *mW, *vW, *mb, *vb, *dWT;
    __nv_bfloat16 *Wb, *Wf;
};

}  // namespace

struct lbm_net {
    lbm_net_config cfg;
    int n, B;  // grid and batch capacity
    int64_t V[3];  // voxels per sample at each level
    Conv conv[kLayers];
    float *Wh, *bh, *gWh, *gbh, *mWh, *vWh, *mbh, *vbh;
    // activations (BF16) and their gradients (FP32)
    __nv_bfloat16 *X0, *A0, *S1, *P1, *A2, *S2, *P2, *A4, *A5, *A6, *C2, *A7, *A8, *C1, *A9, *A10;
    float *dA10, *dA9, *dC1, *dS1, *dA8, *dA7, *dC2, *dS2, *dA6, *dA5, *dA4, *dP2, *dA2, *dP1, *dA0;
    float *out, *dOut, *scal;
    // scratch
    __nv_bfloat16 *xcol, *xcolT, *dZ, *dZT;
    float* y;
    // capacities (elements) of the explicit fallback's scratch: xcol, xcolT, y, dZT
    int64_t xcol_cap, xcolT_cap, y_cap, dzt_cap;
    float* ws;          // split-K partial results of the weight-gradient GEMMs
    size_t ws_floats;
    float* part;        // per-block partial sums of the bias / head gradients
    double* partd;      // per-block partial sums of the loss
    double* loss;
    int* err;
    void* arena;
    size_t arena_bytes;
    int step;
    int implicit;       // convolutions as implicit GEMMs where conv_implicit_supported
    cudaStream_t stream;
    int device;
    int sm_count;
    std::string msg;
};

namespace {

int nfail(lbm_net* N, int code, const char* fmt, const char* detail = nullptr) {
    return record_error(N ? &N->msg : nullptr, code, fmt, detail);
}

#define NET_CUDA(N, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return nfail((N), LBM_ECUDA, "CUDA error in " #call ": %s", cudaGetErrorString(e_)); \
    } while (0)

int pad64(int k) { return (k + 63) / 64 * 64; }

// Layer shapes for channels (c1, c2, c3).
void layer_shapes(const lbm_net_config& c, int cin[kLayers], int cout[kLayers], int level[kLayers]) {
    const int ci[kLayers] = {4, c.c1, c.c1, c.c2, c.c2, c.c3, c.c3, c.c3 + c.c2, c.c2, c.c2 + c.c1, c.c1};
    const int co[kLayers] = {c.c1, c.c1, c.c2, c.c2, c.c3, c.c3, c.c3, c.c2, c.c2, c.c1, c.c1};
    const int lv[kLayers] = {0, 0, 1, 1, 2, 2, 2, 1, 1, 0, 0};
    for (int l = 0; l < kLayers; ++l) {
        cin[l] = ci[l];
        cout[l] = co[l];
        level[l] = lv[l];
    }
}

// splitmix64 (Steele, Lea & Flood 2014) -> uniform (0, 1) -> Box-Muller normal
struct Rng {
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() {
        const double u = uniform(), v = uniform();
        return sqrt(-2.0 * log(u)) * cos(6.283185307179586 * v);
    }
};

struct Carver {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(int64_t count) {
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off = (off + (size_t)count * sizeof(T) + 255) / 256 * 256;
        return p;
    }
};

// K splits of the weight-gradient GEMM of a layer (K = M voxels): about two CTAs per SM
// over the output tiles, at least one K block per split.
int wgrad_splits(const lbm_net* N, const Conv& k, int64_t M) {
    const int tiles = (k.Kp + 127) / 128;
    const int kb = (int)((M + 63) / 64);
    return std::max(1, std::min(2 * N->sm_count / tiles, kb));
}

// Every layer's packing of its FP32 weights into the BF16 operands (one launch).
PackTable pack_table(const lbm_net* N) {
    PackTable t{};
    for (int l = 0; l < kLayers; ++l) {
        const Conv& k = N->conv[l];
        t.seg[l] = PackSeg{k.W, k.cin, k.cs, k.cout, k.Kp, k.Kpf, k.Wb, l == 0 ? nullptr : k.Wf};
    }
    t.count = kLayers;
    return t;
}

// Whether layer k takes the explicit fallback (an im2col matrix and the GEMM) for its
// forward pass, its weight gradient at batch B, its input gradient: the tests conv_fwd and
// conv_bwd make.  The fallback's scratch is sized from these alone.
bool fwd_fallback(const lbm_net* N, const Conv& k) {
    return !(N->implicit && conv_implicit_supported(N->n >> k.level, k.cs, k.cout));
}
bool wgrad_fallback(const lbm_net* N, const Conv& k, int64_t B) {
    return !(N->implicit && conv_wgrad_implicit_supported((int)B, N->n >> k.level, k.cs, k.cout));
}
bool dgrad_fallback(const lbm_net* N, const Conv& k) {
    return !(N->implicit && conv_implicit_supported(N->n >> k.level, k.cout, k.cin));
}

// Lays out (base == nullptr: only sizes) every buffer of the network.
size_t carve(lbm_net* N, char* base) {
    Carver c{base};
    const int64_t B = N->B, V0 = N->V[0], V1 = N->V[1], V2 = N->V[2];
    const int c1 = N->cfg.c1, c2 = N->cfg.c2, c3 = N->cfg.c3;
    int64_t max_y = 0, max_cout = 0;
    int64_t xcol = 0, xcolT = 0, y = 0, dzt = 0;  // the fallback's scratch, where a layer takes it
    size_t ws = 0;
    for (int l = 0; l < kLayers; ++l) {
        Conv& k = N->conv[l];
        const int64_t M = B * N->V[k.level];
        max_y = std::max(max_y, M * k.cout);
        if (fwd_fallback(N, k)) {
            xcol = std::max(xcol, M * k.Kp);
            y = std::max(y, M * k.cout);
        }
        if (wgrad_fallback(N, k, B)) {  // a smaller batch falls back only if this one does
            xcol = std::max(xcol, M * k.Kp);
            xcolT = std::max(xcolT, M * k.Kp);
            dzt = std::max(dzt, M * k.cout);
        }
        if (l > 0 && dgrad_fallback(N, k)) xcol = std::max(xcol, M * k.Kpf);
        max_cout = std::max<int64_t>(max_cout, k.cout);
        // the largest batch asks for the most splits (wgrad_splits grows with M)
        ws = std::max(ws, gemm_splitk_floats(k.Kp, k.cout, (int)M, wgrad_splits(N, k, M)));
        const int64_t w = (int64_t)k.cout * k.K27;
        k.W = c.take<float>(w);
        k.b = c.take<float>(k.cout);
        k.gW = c.take<float>(w);
        k.gb = c.take<float>(k.cout);
        k.mW = c.take<float>(w);
        k.vW = c.take<float>(w);
        k.mb = c.take<float>(k.cout);
        k.vb = c.take<float>(k.cout);
        k.dWT = c.take<float>((int64_t)k.Kp * k.cout);
        k.Wb = c.take<__nv_bfloat16>((int64_t)k.cout * k.Kp);
        k.Wf = c.take<__nv_bfloat16>((int64_t)k.cin * k.Kpf);
    }
    N->Wh = c.take<float>(4 * c1);
    N->bh = c.take<float>(4);
    N->gWh = c.take<float>(4 * c1);
    N->gbh = c.take<float>(4);
    N->mWh = c.take<float>(4 * c1);
    N->vWh = c.take<float>(4 * c1);
    N->mbh = c.take<float>(4);
    N->vbh = c.take<float>(4);
    using bf = __nv_bfloat16;
    N->X0 = c.take<bf>(B * V0 * kX0);
    N->A0 = c.take<bf>(B * V0 * c1);
    N->S1 = c.take<bf>(B * V0 * c1);
    N->P1 = c.take<bf>(B * V1 * c1);
    N->A2 = c.take<bf>(B * V1 * c2);
    N->S2 = c.take<bf>(B * V1 * c2);
    N->P2 = c.take<bf>(B * V2 * c2);
    N->A4 = c.take<bf>(B * V2 * c3);
    N->A5 = c.take<bf>(B * V2 * c3);
    N->A6 = c.take<bf>(B * V2 * c3);
    N->C2 = c.take<bf>(B * V1 * (c3 + c2));
    N->A7 = c.take<bf>(B * V1 * c2);
    N->A8 = c.take<bf>(B * V1 * c2);
    N->C1 = c.take<bf>(B * V0 * (c2 + c1));
    N->A9 = c.take<bf>(B * V0 * c1);
    N->A10 = c.take<bf>(B * V0 * c1);
    N->dA10 = c.take<float>(B * V0 * c1);
    N->dA9 = c.take<float>(B * V0 * c1);
    N->dC1 = c.take<float>(B * V0 * (c2 + c1));
    N->dS1 = c.take<float>(B * V0 * c1);
    N->dA8 = c.take<float>(B * V1 * c2);
    N->dA7 = c.take<float>(B * V1 * c2);
    N->dC2 = c.take<float>(B * V1 * (c3 + c2));
    N->dS2 = c.take<float>(B * V1 * c2);
    N->dA6 = c.take<float>(B * V2 * c3);
    N->dA5 = c.take<float>(B * V2 * c3);
    N->dA4 = c.take<float>(B * V2 * c3);
    N->dP2 = c.take<float>(B * V2 * c2);
    N->dA2 = c.take<float>(B * V1 * c2);
    N->dP1 = c.take<float>(B * V1 * c1);
    N->dA0 = c.take<float>(B * V0 * c1);
    N->out = c.take<float>(B * V0 * 4);
    N->dOut = c.take<float>(B * V0 * 4);
    N->scal = c.take<float>(2 * B);
    N->xcol = c.take<bf>(xcol);
    N->xcolT = c.take<bf>(xcolT);
    N->dZ = c.take<bf>(max_y);
    N->dZT = c.take<bf>(dzt);
    N->y = c.take<float>(y);
    N->xcol_cap = xcol, N->xcolT_cap = xcolT, N->y_cap = y, N->dzt_cap = dzt;
    N->ws = c.take<float>((int64_t)ws);
    N->ws_floats = ws;
    N->part = c.take<float>((int64_t)kMaxPartialBlocks * std::max<int64_t>(max_cout, 4 * c1 + 4));
    N->partd = c.take<double>(kMaxPartialBlocks);
    N->loss = c.take<double>(1);
    return c.off;
}

int conv_fwd(lbm_net* N, int l, const __nv_bfloat16* X, int B, __nv_bfloat16* A) {
    Conv& k = N->conv[l];
    const int n = N->n >> k.level;
    const int64_t M = (int64_t)B * N->V[k.level];
    cudaStream_t st = N->stream;
    if (N->implicit && conv_implicit_supported(n, k.cs, k.cout)) {  // no im2col matrix
        NET_CUDA(N, conv_implicit(X, B, n, k.cs, k.Wb, k.Kp, k.cout, k.b, A, CONV_BIAS_RELU_BF16,
                                  N->err, st));
        return LBM_OK;
    }
    if (M * k.Kp > N->xcol_cap || M * k.cout > N->y_cap)
        return nfail(N, LBM_EINVAL, "internal: the fallback scratch is smaller than the forward pass needs%s");
    NET_CUDA(N, im2col(X, B, n, k.cs, k.Kp, N->xcol, st));
    NET_CUDA(N, gemm_bf16(N->xcol, k.Kp, k.Wb, k.Kp, N->y, k.cout, (int)M, k.cout, k.Kp, GEMM_F32, 1,
                          N->err, st));
    NET_CUDA(N, bias_relu(N->y, k.b, M, k.cout, A, k.cout, 0, st));
    return LBM_OK;
}

// Gradients of layer l given dA (FP32, gradient of its ReLU output A): dW^T and db are
// accumulated; dX (input gradient) is written (plain stores, no atomics) when non-NULL.
int conv_bwd(lbm_net* N, int l, const __nv_bfloat16* X, int B, const __nv_bfloat16* A,
             const float* dA, float* dX) {
    Conv& k = N->conv[l];
    const int n = N->n >> k.level;
    const int64_t M = (int64_t)B * N->V[k.level];
    cudaStream_t st = N->stream;
    NET_CUDA(N, relu_bwd(dA, A, k.cout, 0, M, k.cout, N->dZ, k.gb, N->part, st));
    if (N->implicit && conv_wgrad_implicit_supported(B, n, k.cs, k.cout)) {
        // no im2col matrix and no transpose: both operands read in place
        NET_CUDA(N, conv_wgrad_implicit(X, B, n, k.cs, N->dZ, k.cout, k.Kp, N->ws, N->ws_floats,
                                        wgrad_splits(N, k, M), k.dWT, 0, N->err, st));
    } else {
        if (M * k.Kp > N->xcol_cap || M * k.Kp > N->xcolT_cap || M * k.cout > N->dzt_cap)
            return nfail(N, LBM_EINVAL, "internal: the fallback scratch is smaller than the weight gradient needs%s");
        NET_CUDA(N, cudaMemsetAsync(k.dWT, 0, (size_t)k.Kp * k.cout * 4, st));  // the GEMM adds
        NET_CUDA(N, transpose(N->dZ, M, k.cout, k.cout, N->dZT, M, st));
        if (im2colT_supported(n, k.cs, M)) {  // written transposed: no im2col matrix in between
            NET_CUDA(N, im2colT(X, B, n, k.cs, k.Kp, N->xcolT, st));
        } else {
            NET_CUDA(N, im2col(X, B, n, k.cs, k.Kp, N->xcol, st));
            NET_CUDA(N, transpose(N->xcol, M, k.Kp, k.Kp, N->xcolT, M, st));
        }
        NET_CUDA(N, gemm_bf16_add_splitk(N->xcolT, M, N->dZT, M, k.dWT, k.cout, k.Kp, k.cout, (int)M,
                                         wgrad_splits(N, k, M), N->ws, N->ws_floats, N->err, st));
    }
    if (dX) {  // dX = im2col(dZ) Wf^T: the convolution of dZ with the mirrored weights
        if (N->implicit && conv_implicit_supported(n, k.cout, k.cin)) {
            NET_CUDA(N, conv_implicit(N->dZ, B, n, k.cout, k.Wf, k.Kpf, k.cin, nullptr, dX, CONV_F32,
                                      N->err, st));
        } else {  // the xcol scratch is free again
            if (M * k.Kpf > N->xcol_cap)
                return nfail(N, LBM_EINVAL, "internal: the fallback scratch is smaller than the input gradient needs%s");
            NET_CUDA(N, im2col(N->dZ, B, n, k.cout, k.Kpf, N->xcol, st));
            NET_CUDA(N, gemm_bf16(N->xcol, k.Kpf, k.Wf, k.Kpf, dX, k.cin, (int)M, k.cin, k.Kpf,
                                  GEMM_F32, 1, N->err, st));
        }
    }
    return LBM_OK;
}

#define NET_RC(x)                 \
    do {                          \
        int rc_ = (x);            \
        if (rc_ != LBM_OK) return rc_; \
    } while (0)

int forward(lbm_net* N, int B) {
    cudaStream_t st = N->stream;
    const int n = N->n, c1 = N->cfg.c1, c2 = N->cfg.c2, c3 = N->cfg.c3;
    const int64_t M1 = (int64_t)B * N->V[1];
    NET_CUDA(N, features(B, n, N->scal, N->X0, kX0, st));
    NET_RC(conv_fwd(N, 0, N->X0, B, N->A0));
    NET_RC(conv_fwd(N, 1, N->A0, B, N->S1));
    NET_CUDA(N, avgpool(N->S1, B, n, c1, N->P1, st));
    NET_RC(conv_fwd(N, 2, N->P1, B, N->A2));
    NET_RC(conv_fwd(N, 3, N->A2, B, N->S2));
    NET_CUDA(N, avgpool(N->S2, B, n / 2, c2, N->P2, st));
    NET_RC(conv_fwd(N, 4, N->P2, B, N->A4));
    NET_RC(conv_fwd(N, 5, N->A4, B, N->A5));
    NET_RC(conv_fwd(N, 6, N->A5, B, N->A6));
    NET_CUDA(N, upsample(N->A6, B, n / 2, c3, N->C2, c3 + c2, 0, st));
    NET_CUDA(N, copy_channels(N->S2, M1, c2, N->C2, c3 + c2, c3, st));
    NET_RC(conv_fwd(N, 7, N->C2, B, N->A7));
    NET_RC(conv_fwd(N, 8, N->A7, B, N->A8));
    NET_CUDA(N, upsample(N->A8, B, n, c2, N->C1, c2 + c1, 0, st));
    NET_CUDA(N, copy_channels(N->S1, (int64_t)B * N->V[0], c1, N->C1, c2 + c1, c2, st));
    NET_RC(conv_fwd(N, 9, N->C1, B, N->A9));
    NET_RC(conv_fwd(N, 10, N->A9, B, N->A10));
    NET_CUDA(N, head_fwd(N->A10, (int64_t)B * N->V[0], c1, N->Wh, N->bh, N->out, st));
    return LBM_OK;
}

// Loss and every parameter gradient for the batch (forward must have run).
int backward(lbm_net* N, int B, const float* target) {
    cudaStream_t st = N->stream;
    const int n = N->n, c1 = N->cfg.c1, c2 = N->cfg.c2, c3 = N->cfg.c3;
    const int64_t M0 = (int64_t)B * N->V[0], M1 = (int64_t)B * N->V[1];
    // every gradient below is stored (not added) by its one producer: no zeroing pass
    NET_CUDA(N, mse(N->out, target, M0 * 4, N->dOut, N->loss, N->partd, st));
    NET_CUDA(N, head_bwd(N->dOut, N->A10, M0, c1, N->Wh, N->dA10, N->gWh, N->gbh, N->part, st));
    NET_RC(conv_bwd(N, 10, N->A9, B, N->A10, N->dA10, N->dA9));
    NET_RC(conv_bwd(N, 9, N->C1, B, N->A9, N->dA9, N->dC1));
    NET_CUDA(N, upsample_bwd(N->dC1, c2 + c1, 0, B, n, c2, N->dA8, st));
    NET_CUDA(N, slice_grad(N->dC1, c2 + c1, c2, M0, c1, N->dS1, 0, st));
    NET_RC(conv_bwd(N, 8, N->A7, B, N->A8, N->dA8, N->dA7));
    NET_RC(conv_bwd(N, 7, N->C2, B, N->A7, N->dA7, N->dC2));
    NET_CUDA(N, upsample_bwd(N->dC2, c3 + c2, 0, B, n / 2, c3, N->dA6, st));
    NET_CUDA(N, slice_grad(N->dC2, c3 + c2, c3, M1, c2, N->dS2, 0, st));
    NET_RC(conv_bwd(N, 6, N->A5, B, N->A6, N->dA6, N->dA5));
    NET_RC(conv_bwd(N, 5, N->A4, B, N->A5, N->dA5, N->dA4));
    NET_RC(conv_bwd(N, 4, N->P2, B, N->A4, N->dA4, N->dP2));
    NET_CUDA(N, avgpool_bwd(N->dP2, B, n / 2, c2, N->dS2, 1, st));
    NET_RC(conv_bwd(N, 3, N->A2, B, N->S2, N->dS2, N->dA2));
    NET_RC(conv_bwd(N, 2, N->P1, B, N->A2, N->dA2, N->dP1));
    NET_CUDA(N, avgpool_bwd(N->dP1, B, n, c1, N->dS1, 1, st));
    NET_RC(conv_bwd(N, 1, N->A0, B, N->S1, N->dS1, N->dA0));
    NET_RC(conv_bwd(N, 0, N->X0, B, N->A0, N->dA0, nullptr));
    UnpackTable t{};
    for (int l = 0; l < kLayers; ++l) {
        const Conv& k = N->conv[l];
        t.seg[l] = UnpackSeg{k.dWT, k.cout, k.cin, k.cs, k.gW};
    }
    t.count = kLayers;
    NET_CUDA(N, unpack_grad(t, st));
    return LBM_OK;
}

int update(lbm_net* N) {
    cudaStream_t st = N->stream;
    const lbm_net_config& c = N->cfg;
    N->step += 1;
    AdamTable t{};
    int i = 0;
    for (int l = 0; l < kLayers; ++l) {
        Conv& k = N->conv[l];
        t.seg[i++] = AdamSeg{k.W, k.gW, k.mW, k.vW, (int64_t)k.cout * k.K27};
        t.seg[i++] = AdamSeg{k.b, k.gb, k.mb, k.vb, (int64_t)k.cout};
    }
    t.seg[i++] = AdamSeg{N->Wh, N->gWh, N->mWh, N->vWh, (int64_t)4 * c.c1};
    t.seg[i++] = AdamSeg{N->bh, N->gbh, N->mbh, N->vbh, 4};
    t.count = i;
    NET_CUDA(N, adam(t, c.lr, c.beta1, c.beta2, c.eps, N->step, st));
    NET_CUDA(N, pack_weights(pack_table(N), st));
    return LBM_OK;
}

int wait_net(lbm_net* N) {
    int rc = wait_stream_for(N->stream, 600.0, &N->msg);
    if (rc != LBM_OK) return rc;
    int h = 0;
    NET_CUDA(N, cudaMemcpy(&h, N->err, sizeof h, cudaMemcpyDeviceToHost));
    if (h) {
        cudaMemset(N->err, 0, sizeof(int));
        return nfail(N, LBM_ETIMEOUT, "a wait inside a tensor-core kernel timed out%s");
    }
    return LBM_OK;
}

// The bounded wait (and the kernels' error word) first, then the loss into caller memory:
// a copy into pageable memory issued before the wait would block without a time limit.
int finish_with_loss(lbm_net* N, double* loss) {
    int rc = wait_net(N);
    if (rc != LBM_OK || !loss) return rc;
    NET_CUDA(N, cudaMemcpy(loss, N->loss, 8, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int upload_scalars(lbm_net* N, int B, const float* scalars) {
    if (B < 1 || B > N->B || !scalars) return nfail(N, LBM_EINVAL, "batch outside 1..max_batch or NULL scalars%s");
    NET_CUDA(N, cudaMemcpyAsync(N->scal, scalars, (size_t)2 * B * sizeof(float), cudaMemcpyHostToDevice,
                                N->stream));
    return LBM_OK;
}

// Flattened parameter (or gradient) layout: per layer W [cout][27 cin] then b; then the
// head W [4][c1] and b [4].
template <typename Fn>
void for_each_param(lbm_net* N, bool grads, Fn&& fn) {
    for (int l = 0; l < kLayers; ++l) {
        Conv& k = N->conv[l];
        fn(grads ? k.gW : k.W, (int64_t)k.cout * k.K27);
        fn(grads ? k.gb : k.b, (int64_t)k.cout);
    }
    fn(grads ? N->gWh : N->Wh, (int64_t)4 * N->cfg.c1);
    fn(grads ? N->gbh : N->bh, (int64_t)4);
}

}  // namespace

extern "C" void lbm_net_default_config(lbm_net_config* c) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->n = 64;
    c->max_batch = 2;
    c->c1 = 32;
    c->c2 = 64;
    c->c3 = 128;
    c->seed = 1;
    c->lr = 1e-3f;
    c->beta1 = 0.9f;
    c->beta2 = 0.999f;
    c->eps = 1e-8f;
    c->cuda_stream = nullptr;
}

extern "C" void lbm_net_destroy(lbm_net* N) {
    if (!N) return;
    wait_stream_for(N->stream, 600.0, nullptr);
    if (N->arena) cudaFree(N->arena);
    delete N;
}

extern "C" int lbm_net_create(const lbm_net_config* cfg, lbm_net** out) {
    if (!out) return nfail(nullptr, LBM_EINVAL, "out is NULL%s");
    *out = nullptr;
    lbm_net_config c;
    if (cfg) c = *cfg; else lbm_net_default_config(&c);
    if (c.n < 8 || c.n % 8 || c.n > 256 || c.max_batch < 1 || c.c1 < 8 || c.c1 % 8 || c.c1 > 64 ||
        c.c2 % 8 || c.c2 < 8 || c.c2 > 256 || c.c3 % 8 || c.c3 < 8 || c.c3 > 256 || !(c.lr > 0))
        return nfail(nullptr, LBM_EINVAL,
                     "invalid network: n a multiple of 8 in 8..256, channels multiples of 8 "
                     "(c1 <= 64, c2, c3 <= 256), max_batch >= 1%s");
    const double M0 = (double)c.max_batch * c.n * c.n * c.n;
    if (M0 > 2.0e9)  // GEMM rows and the weight-gradient K are 32-bit
        return nfail(nullptr, LBM_EINVAL, "n^3 * max_batch must stay below 2^31%s");
    lbm_net* N = new (std::nothrow) lbm_net();
    if (!N) return nfail(nullptr, LBM_ENOMEM, "host allocation failed%s");
    N->cfg = c;
    N->n = c.n;
    N->B = c.max_batch;
    N->implicit = 1;
    N->stream = static_cast<cudaStream_t>(c.cuda_stream);
    for (int lv = 0; lv < 3; ++lv) {
        const int64_t m = c.n >> lv;
        N->V[lv] = m * m * m;
    }
    int cin[kLayers], cout[kLayers], level[kLayers];
    layer_shapes(c, cin, cout, level);
    for (int l = 0; l < kLayers; ++l) {
        Conv& k = N->conv[l];
        k.cin = cin[l];
        k.cout = cout[l];
        k.level = level[l];
        k.K27 = 27 * cin[l];
        k.cs = l == 0 ? kX0 : cin[l];
        k.Kp = pad64(27 * k.cs);
        k.Kpf = pad64(27 * cout[l]);
    }
    if (cudaGetDevice(&N->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&N->sm_count, cudaDevAttrMultiProcessorCount, N->device) != cudaSuccess) {
        delete N;
        return nfail(nullptr, LBM_ECUDA, "no CUDA device%s");
    }
    N->arena_bytes = carve(N, nullptr);
    cudaError_t e = cudaMalloc(&N->arena, N->arena_bytes);
    if (e != cudaSuccess) {
        delete N;
        return nfail(nullptr, LBM_ENOMEM, "cudaMalloc of the network failed: %s", cudaGetErrorString(e));
    }
    carve(N, static_cast<char*>(N->arena));
    e = cudaMalloc(&N->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(N->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(N->arena, 0, N->arena_bytes);  // zero moments
    if (e != cudaSuccess) {
        lbm_net_destroy(N);
        return nfail(nullptr, LBM_ECUDA, "cudaMalloc / cudaMemset failed%s");
    }
    // He-normal weights (std sqrt(2 / fan_in)), zero biases; head std sqrt(1 / c1) / 4
    Rng rng{c.seed};
    std::vector<float> host;
    int rc = LBM_OK;
    for (int l = 0; l < kLayers && rc == LBM_OK; ++l) {
        Conv& k = N->conv[l];
        const double sd = sqrt(2.0 / k.K27);
        host.resize((size_t)k.cout * k.K27);
        for (auto& w : host) w = (float)(sd * rng.normal());
        if (cudaMemcpy(k.W, host.data(), host.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = nfail(N, LBM_ECUDA, "weight upload failed%s");
    }
    if (rc == LBM_OK && pack_weights(pack_table(N), N->stream) != cudaSuccess)
        rc = nfail(N, LBM_ECUDA, "weight packing failed%s");
    if (rc == LBM_OK) {
        host.resize((size_t)4 * c.c1);
        const double sd = 0.25 * sqrt(1.0 / c.c1);
        for (auto& w : host) w = (float)(sd * rng.normal());
        if (cudaMemcpy(N->Wh, host.data(), host.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = nfail(N, LBM_ECUDA, "weight upload failed%s");
    }
    if (rc == LBM_OK) rc = wait_net(N);
    if (rc != LBM_OK) {
        std::string m = N->msg;
        lbm_net_destroy(N);
        set_last_error(m.c_str());
        return rc;
    }
    *out = N;
    return LBM_OK;
}

extern "C" int64_t lbm_net_param_count(const lbm_net* N) {
    if (!N) return 0;
    int64_t total = 0;
    for_each_param(const_cast<lbm_net*>(N), false, [&](float*, int64_t n) { total += n; });
    return total;
}

extern "C" int lbm_net_get_params(lbm_net* N, float* host, int64_t count, int grads) {
    if (!N || !host || count != lbm_net_param_count(N)) return nfail(N, LBM_EINVAL, "NULL or wrong count%s");
    int rc = wait_net(N);
    if (rc != LBM_OK) return rc;
    int64_t off = 0;
    cudaError_t e = cudaSuccess;
    for_each_param(N, grads != 0, [&](float* dev, int64_t n) {
        if (e == cudaSuccess) e = cudaMemcpy(host + off, dev, (size_t)n * 4, cudaMemcpyDeviceToHost);
        off += n;
    });
    NET_CUDA(N, e);
    return LBM_OK;
}

extern "C" int lbm_net_set_params(lbm_net* N, const float* host, int64_t count) {
    if (!N || !host || count != lbm_net_param_count(N)) return nfail(N, LBM_EINVAL, "NULL or wrong count%s");
    int rc = wait_net(N);
    if (rc != LBM_OK) return rc;
    int64_t off = 0;
    cudaError_t e = cudaSuccess;
    for_each_param(N, false, [&](float* dev, int64_t n) {
        if (e == cudaSuccess) e = cudaMemcpy(dev, host + off, (size_t)n * 4, cudaMemcpyHostToDevice);
        off += n;
    });
    NET_CUDA(N, e);
    NET_CUDA(N, pack_weights(pack_table(N), N->stream));
    return wait_net(N);
}

extern "C" int lbm_net_forward(lbm_net* N, int batch, const float* scalars, float* out) {
    if (!N || !out) return nfail(N, LBM_EINVAL, "NULL argument%s");
    NET_RC(upload_scalars(N, batch, scalars));
    NET_RC(forward(N, batch));
    NET_CUDA(N, cudaMemcpyAsync(out, N->out, (size_t)batch * N->V[0] * 4 * sizeof(float),
                                cudaMemcpyDeviceToDevice, N->stream));
    return wait_net(N);
}

extern "C" int lbm_net_gradients(lbm_net* N, int batch, const float* scalars, const float* targets,
                                 double* loss) {
    if (!N || !targets) return nfail(N, LBM_EINVAL, "NULL argument%s");
    NET_RC(upload_scalars(N, batch, scalars));
    NET_RC(forward(N, batch));
    NET_RC(backward(N, batch, targets));
    return finish_with_loss(N, loss);
}

extern "C" int lbm_net_train_step(lbm_net* N, int batch, const float* scalars, const float* targets,
                                  double* loss) {
    if (!N || !targets) return nfail(N, LBM_EINVAL, "NULL argument%s");
    NET_RC(upload_scalars(N, batch, scalars));
    NET_RC(forward(N, batch));
    NET_RC(backward(N, batch, targets));
    NET_RC(update(N));
    return finish_with_loss(N, loss);
}

extern "C" int lbm_net_set_lr(lbm_net* N, float lr) {
    if (!N || !(lr > 0)) return nfail(N, LBM_EINVAL, "NULL network or lr <= 0%s");
    N->cfg.lr = lr;
    return LBM_OK;
}

extern "C" void lbm_net_encode(double Ra, double Pr, float* out2) {
    if (!out2) return;
    out2[0] = (float)((log10(Ra) - 4.5) / 1.5);
    out2[1] = (float)((log10(Pr) - 0.345) / 0.5);
}

extern "C" const char* lbm_net_last_error(const lbm_net* N) {
    return N ? N->msg.c_str() : lbm_last_error(nullptr);
}

extern "C" int lbm_net_tensor(lbm_net* N, int which, int batch, void* host, int64_t count) {
    if (!N || !host || batch < 1 || batch > N->B) return nfail(N, LBM_EINVAL, "NULL argument or batch outside 1..max_batch%s");
    const int c1 = N->cfg.c1, c2 = N->cfg.c2, c3 = N->cfg.c3;
    struct T { const void* p; int level, channels, bytes, ld; };
    const T t[LBM_NET_TENSORS] = {
        {N->X0, 0, 4, 2, kX0}, {N->A0, 0, c1, 2}, {N->S1, 0, c1, 2}, {N->P1, 1, c1, 2},
        {N->A2, 1, c2, 2}, {N->S2, 1, c2, 2}, {N->P2, 2, c2, 2}, {N->A4, 2, c3, 2},
        {N->A5, 2, c3, 2}, {N->A6, 2, c3, 2}, {N->C2, 1, c3 + c2, 2}, {N->A7, 1, c2, 2},
        {N->A8, 1, c2, 2}, {N->C1, 0, c2 + c1, 2}, {N->A9, 0, c1, 2}, {N->A10, 0, c1, 2},
        {N->out, 0, 4, 4},
        {N->dA10, 0, c1, 4}, {N->dA9, 0, c1, 4}, {N->dC1, 0, c2 + c1, 4}, {N->dS1, 0, c1, 4},
        {N->dA8, 1, c2, 4}, {N->dA7, 1, c2, 4}, {N->dC2, 1, c3 + c2, 4}, {N->dS2, 1, c2, 4},
        {N->dA6, 2, c3, 4}, {N->dA5, 2, c3, 4}, {N->dA4, 2, c3, 4}, {N->dP2, 2, c2, 4},
        {N->dA2, 1, c2, 4}, {N->dP1, 1, c1, 4}, {N->dA0, 0, c1, 4}, {N->dOut, 0, 4, 4},
    };
    if (which < 0 || which >= LBM_NET_TENSORS) return nfail(N, LBM_EINVAL, "unknown tensor id%s");
    const T& d = t[which];
    const int64_t elems = (int64_t)batch * N->V[d.level] * d.channels;
    if (count != elems) return nfail(N, LBM_EINVAL, "count differs from batch * voxels * channels%s");
    int rc = wait_net(N);  // bounded, before the copy into caller memory
    if (rc != LBM_OK) return rc;
    if (d.ld > d.channels)  // a padded row: its first `channels` values
        NET_CUDA(N, cudaMemcpy2D(host, (size_t)d.channels * d.bytes, d.p, (size_t)d.ld * d.bytes,
                                 (size_t)d.channels * d.bytes, (size_t)(elems / d.channels),
                                 cudaMemcpyDeviceToHost));
    else
        NET_CUDA(N, cudaMemcpy(host, d.p, (size_t)elems * d.bytes, cudaMemcpyDeviceToHost));
    return LBM_OK;
}
