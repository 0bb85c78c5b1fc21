"""The warm-start network's CUDA kernels (include/lbm_net.h) against the FP64 CPU oracle:
the tensor-core GEMM first.

GEMM tolerance: the operands are BF16 (exactly representable inputs on both sides) and
the products are accumulated in FP32, so |C - C_fp64| <= 2^-22 * K * sum_k |a_k b_k| per
element bounds the accumulation error with a wide margin (written below as 1e-6 * K).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def torch_mod():
    import torch
    return torch


def bf16_pair(shape_a, shape_b, seed):
    torch = torch_mod()
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(shape_a, generator=g, dtype=torch.float64).to(torch.bfloat16)
    B = torch.randn(shape_b, generator=g, dtype=torch.float64).to(torch.bfloat16)
    return A, B


def reference(A, B):
    a = A.double().numpy()
    b = B.double().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 64, 128), (300, 100, 200),
                                   (1024, 256, 1024), (130, 16, 72), (512, 200, 640),
                                   (4096, 128, 1728)])
def test_gemm_f32_against_fp64(M, N, K):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    Kp = (K + 7) // 8 * 8
    A, B = bf16_pair((M, Kp), (N, Kp), M + N + K)
    A[:, K:] = 0
    B[:, K:] = 0
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32, K=K)
    ref, mag = reference(A[:, :K], B[:, :K])
    got = C.cpu().double().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= 1e-6 * K * mag + 1e-30).all()


def test_gemm_bf16_output_and_strided_operands():
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    A, B = bf16_pair((384, 256), (96, 256), 7)
    Ad, Bd = A.cuda(), B.cuda()
    # operand views with row strides 256 over K = 192, and an output with row stride 128
    C = torch.zeros((384, 128), dtype=torch.bfloat16, device="cuda")
    net.gemm_bf16(Ad[:, :192], Bd[:, :192], C[:, :96], net.GEMM_BF16, K=192)
    ref, _ = reference(A[:, :192], B[:, :192])
    got = C[:, :96].cpu().double().numpy()
    assert np.allclose(got, ref, rtol=2 ** -7, atol=1e-2)
    assert (C[:, 96:] == 0).all()


@pytest.mark.parametrize("splits", [1, 3, 8])
def test_gemm_split_k_accumulates(splits):
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    M, N, K = 256, 64, 64 * 20
    A, B = bf16_pair((M, K), (N, K), 11)
    C = torch.ones((M, N), dtype=torch.float32, device="cuda")
    net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32_ADD, splits=splits)
    ref, mag = reference(A, B)
    got = C.cpu().double().numpy() - 1.0
    assert (np.abs(got - ref) <= 1e-6 * K * mag + 1e-6).all()


def test_gemm_rejects_bad_arguments():
    torch = torch_mod()
    from paper_1710_04751_gb300 import net
    from paper_1710_04751_gb300.lbm import LBMError
    A, B = bf16_pair((128, 128), (32, 128), 3)
    C = torch.zeros((128, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(LBMError):  # split K (two K blocks) without accumulation
        net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32, splits=2)
    with pytest.raises(LBMError):  # row stride not a multiple of 8
        At = torch.zeros((128, 70), dtype=torch.bfloat16, device="cuda")
        net.gemm_bf16(At, B.cuda(), C, net.GEMM_F32, K=64)
