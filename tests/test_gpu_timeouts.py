"""Bounded waits run out without faulting or hanging the GPU, and leave everything usable.

* A context whose wait bound is set to 1e-9 s returns LBM_ETIMEOUT from an lbm_step that
  ends with a residual check while its kernels are still running, and from the calls
  that read results before the GPU is done; once lbm_synchronize reports the stream idle,
  the same context gives the state a context that never timed out has.
* The tensor-core GEMM's in-kernel wait: the diagnostic launch withholds the operand
  loads, so its bounded wait (10 ms) runs out; the call returns LBM_ETIMEOUT, and the next
  GEMM is exact again."""
import math
import time

import numpy as np
import pytest

from paper_1710_04751_gb300.lbm import LBM_ETIMEOUT

pytestmark = pytest.mark.gpu


def _cavity(lbm):
    return lbm.LBM((128, 128, 128), 15, Ra=1e5, Pr=0.71, Ma=0.05 * math.sqrt(3.0),
                   precision=lbm.FP32, residual_interval=100)


def test_host_wait_times_out_and_the_context_recovers():
    import paper_1710_04751_gb300 as lbm
    a, b = _cavity(lbm), _cavity(lbm)
    a.set_timeout(1e-9)
    with pytest.raises(lbm.LBMError) as e:
        a.step(2000)  # ~0.16 s of kernels; the residual check's wait runs out at once
    assert e.value.code == LBM_ETIMEOUT
    with pytest.raises(lbm.LBMError) as e:
        a.nusselt()  # waits before copying: times out again, copies nothing
    assert e.value.code == LBM_ETIMEOUT
    t0 = time.time()
    while True:  # the queued work keeps running; poll until the stream is idle
        try:
            a.synchronize()
            break
        except lbm.LBMError as err:
            assert err.code == LBM_ETIMEOUT
            assert time.time() - t0 < 60
    a.set_timeout(600.0)
    assert a.steps_done == 2000
    b.step(2000)
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.nusselt() == b.nusselt()
    a.step(100)  # and it keeps stepping
    assert a.residual() >= 0
    with pytest.raises(lbm.LBMError):
        a.set_timeout(0.0)
    a.close()
    b.close()


def test_gemm_bounded_wait_runs_out_and_the_next_gemm_is_exact():
    import torch
    import paper_1710_04751_gb300 as lbm
    from paper_1710_04751_gb300 import net
    for _ in range(2):
        assert net.gemm_timeout_probe() == LBM_ETIMEOUT
    g = torch.Generator().manual_seed(3)
    A = torch.randn((256, 128), generator=g, dtype=torch.float64).to(torch.bfloat16)
    B = torch.randn((64, 128), generator=g, dtype=torch.float64).to(torch.bfloat16)
    C = torch.full((256, 64), float("nan"), dtype=torch.float32, device="cuda")
    net.gemm_bf16(A.cuda(), B.cuda(), C, net.GEMM_F32)
    a, b = A.double().numpy(), B.double().numpy()
    ref, mag = a @ b.T, np.abs(a) @ np.abs(b).T
    got = C.cpu().double().numpy()
    assert (np.abs(got - ref) <= 1e-6 * 128 * mag).all()
