"""Python binding of include/lbm_net.h (argument marshalling only): the tensor-core GEMM
building block and the learned warm-start network.  Tensors are torch CUDA tensors;
every computation runs in liblbm.so."""
import ctypes

from .lbm import LBM_OK, LBMError, load

GEMM_F32, GEMM_BF16, GEMM_F32_ADD = 0, 1, 2

# Every entry point include/lbm_net.h declares (checked by tests/test_abi.py).
EXPORTS = (
    "lbm_nn_gemm_bf16",
)

_bound = False


def _lib():
    global _bound
    L = load()
    if _bound:
        return L
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.lbm_nn_gemm_bf16.argtypes = [vp, i64, vp, i64, vp, i64, i32, i32, i32, i32, i32, vp]
    _bound = True
    return L


def _check(rc):
    if rc != LBM_OK:
        raise LBMError(rc, _lib().lbm_last_error(None).decode())


def _stream(t):
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def gemm_bf16(A, B, C, out_mode=GEMM_F32, splits=1, K=None):
    """C[M][N] (=, or += with GEMM_F32_ADD) A[M][K] @ B[N][K]^T; A, B bfloat16 CUDA
    tensors (row strides multiples of 8), C float32 or bfloat16."""
    M, N = C.shape
    K = A.shape[1] if K is None else K
    _check(_lib().lbm_nn_gemm_bf16(A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0),
                                   C.data_ptr(), C.stride(0), M, N, K, out_mode, splits,
                                   _stream(C)))
