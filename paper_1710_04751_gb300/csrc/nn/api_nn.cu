// api_nn.cu -- the C ABI of include/lbm_net.h.
#include <mutex>

#include "../context.h"
#include "lbm_net.h"
#include "nn.h"

using namespace lbm;

namespace {

// Per-device error word the network kernels write on a timeout.
__device__ int nn_error_word;

// Operand and output of the timeout diagnostic (nothing reads the operand; nothing is
// stored to the output).
__device__ __align__(128) __nv_bfloat16 nn_probe_operand[128 * 64];
__device__ __align__(128) float nn_probe_out[128 * 32];

int* error_word() {
    static int* ptr[64] = {};
    static std::mutex mu;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, nn_error_word) != cudaSuccess) return nullptr;
        ptr[dev] = static_cast<int*>(p);
    }
    return ptr[dev];
}

// Waits for the stream and turns a recorded kernel timeout into LBM_ETIMEOUT.
int finish(cudaStream_t st, int* err) {
    int rc = wait_stream_for(st, 600.0, nullptr);
    if (rc != LBM_OK) return rc;
    int h = 0;
    if (cudaMemcpy(&h, err, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess)
        return record_error(nullptr, LBM_ECUDA, "reading the network error word failed%s");
    if (h != 0) {
        cudaMemset(err, 0, sizeof(int));
        return record_error(nullptr, LBM_ETIMEOUT, "a wait inside a tensor-core kernel timed out%s");
    }
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_nn_gemm_bf16(const void* A, int64_t lda, const void* B, int64_t ldb, void* C,
                                int64_t ldc, int M, int N, int K, int out_mode, int splits,
                                void* cuda_stream) {
    if (!A || !B || !C || ldc < N)
        return record_error(nullptr, LBM_EINVAL, "NULL operand or ldc < N%s");
    // the public modes only (the internal split-slice mode writes past C)
    if (out_mode != LBM_GEMM_F32 && out_mode != LBM_GEMM_BF16 && out_mode != LBM_GEMM_F32_ADD)
        return record_error(nullptr, LBM_EINVAL, "invalid GEMM mode%s");
    int* err = error_word();
    if (!err) return record_error(nullptr, LBM_ECUDA, "no CUDA device%s");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = nn::gemm_bf16(static_cast<const __nv_bfloat16*>(A), lda,
                                        static_cast<const __nv_bfloat16*>(B), ldb, C, ldc, M, N, K,
                                        out_mode, splits, err, st);
    if (e == cudaErrorInvalidValue)
        return record_error(nullptr, LBM_EINVAL, "invalid GEMM shape, stride, alignment or mode%s");
    if (e != cudaSuccess) return record_error(nullptr, LBM_ECUDA, "GEMM launch failed: %s", cudaGetErrorString(e));
    return finish(st, err);
}

extern "C" int lbm_nn_gemm_timeout_probe(void* cuda_stream) {
    int* err = error_word();
    if (!err) return record_error(nullptr, LBM_ECUDA, "no CUDA device%s");
    void* op = nullptr;
    void* out = nullptr;
    if (cudaGetSymbolAddress(&op, nn_probe_operand) != cudaSuccess ||
        cudaGetSymbolAddress(&out, nn_probe_out) != cudaSuccess)
        return record_error(nullptr, LBM_ECUDA, "cannot address the diagnostic buffers%s");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // earlier work on the stream must not be mistaken for the probe's own timeout
    int rc = finish(st, err);
    if (rc != LBM_OK) return rc;
    const cudaError_t e = nn::gemm_timeout_probe(static_cast<const __nv_bfloat16*>(op),
                                                 static_cast<float*>(out), err, st);
    if (e != cudaSuccess)
        return record_error(nullptr, LBM_ECUDA, "probe launch failed: %s", cudaGetErrorString(e));
    return finish(st, err);  // LBM_ETIMEOUT when the bounded wait ran out as intended
}

extern "C" int lbm_nn_conv3d_wgrad_bf16(const void* X, int batch, int n, int cin, const void* dZ, int cout,
                                        int Kp, float* ws, int64_t ws_floats, int splits, float* dWT,
                                        void* cuda_stream) {
    if (!X || !dZ || !ws || !dWT) return record_error(nullptr, LBM_EINVAL, "NULL operand%s");
    if (!nn::conv_wgrad_implicit_supported(batch, n, cin, cout) || Kp < 27 * cin || splits < 1 || ws_floats < 0)
        return record_error(nullptr, LBM_EINVAL,
                            "implicit weight gradient needs n a power of two in 2..256, cin a multiple of 32, "
                            "cout a multiple of 8 in 8..256, Kp >= 27 cin and splits >= 1%s");
    int* err = error_word();
    if (!err) return record_error(nullptr, LBM_ECUDA, "no CUDA device%s");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = nn::conv_wgrad_implicit(static_cast<const __nv_bfloat16*>(X), batch, n, cin,
                                                  static_cast<const __nv_bfloat16*>(dZ), cout, Kp, ws,
                                                  (size_t)ws_floats, splits, dWT, 1, err, st);
    if (e == cudaErrorInvalidValue)
        return record_error(nullptr, LBM_EINVAL, "invalid weight-gradient shape, workspace or alignment%s");
    if (e != cudaSuccess)
        return record_error(nullptr, LBM_ECUDA, "weight-gradient launch failed: %s", cudaGetErrorString(e));
    return finish(st, err);
}

extern "C" int lbm_nn_conv3d_bf16(const void* X, int batch, int n, int cin, const void* W,
                                  int64_t ldw, int cout, const float* bias, void* out, int mode,
                                  void* cuda_stream) {
    if (!X || !W || !out || (mode == LBM_CONV_BIAS_RELU_BF16 && !bias))
        return record_error(nullptr, LBM_EINVAL, "NULL operand%s");
    if (mode != LBM_CONV_BIAS_RELU_BF16 && mode != LBM_CONV_F32)
        return record_error(nullptr, LBM_EINVAL, "invalid convolution mode%s");
    if (!nn::conv_implicit_supported(n, cin, cout) || batch < 1)
        return record_error(nullptr, LBM_EINVAL,
                            "implicit convolution needs cin a multiple of 32, n a power of two in 2..256, "
                            "1 <= cout <= 256 and batch >= 1%s");
    int* err = error_word();
    if (!err) return record_error(nullptr, LBM_ECUDA, "no CUDA device%s");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const cudaError_t e = nn::conv_implicit(
        static_cast<const __nv_bfloat16*>(X), batch, n, cin, static_cast<const __nv_bfloat16*>(W), ldw,
        cout, bias, out, mode == LBM_CONV_BIAS_RELU_BF16 ? nn::CONV_BIAS_RELU_BF16 : nn::CONV_F32, err, st);
    if (e == cudaErrorInvalidValue)
        return record_error(nullptr, LBM_EINVAL, "invalid convolution shape, stride or alignment%s");
    if (e != cudaSuccess)
        return record_error(nullptr, LBM_ECUDA, "convolution launch failed: %s", cudaGetErrorString(e));
    return finish(st, err);
}

