"""lbm_nusselt_noalloc: the allocation-free Nusselt reduction for callers that cannot
call cudaMalloc (their device memory is owned by an enclosing application, or they must
not allocate once running).  Through the C ABI, on populations held in caller-owned
device buffers, it must return what lbm_nusselt returns for the same state, on two calls
in a row (the static scratch is reused) and again after the state has changed.

Collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

VALUE_KEYS = ("hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_min", "umax", "wmax")
POS_KEYS = ("mid_max_z", "mid_min_z", "umax_z", "wmax_x")


def _device_copy(torch, arr, dtype):
    return torch.from_numpy(np.ascontiguousarray(arr)).to(device="cuda", dtype=dtype).contiguous()


def _check(got, expect):
    for k in VALUE_KEYS:
        assert got[k] == pytest.approx(expect[k], rel=1e-12, abs=1e-14), k
    for k in POS_KEYS:
        assert got[k] == expect[k], k


@pytest.mark.parametrize("q,prec", [(15, "FP32"), (7, "FP32"), (15, "FP64")])
def test_noalloc_nusselt_matches_lbm_nusselt(q, prec):
    import torch

    import paper_1710_04751_gb300 as lbm

    precision = getattr(lbm, prec)
    dtype = torch.float32 if precision == lbm.FP32 else torch.float64
    grid = (24, 20, 18)
    ncell = grid[0] * grid[1] * grid[2]
    sim = lbm.LBM(grid, q, Ra=2e3, precision=precision)
    params = sim.params_struct()
    stream = torch.cuda.current_stream().cuda_stream
    for advance in (150, 250):
        sim.step(advance)
        expect = sim.nusselt()
        f, g = sim.get_populations()  # the stored state, exactly (FP32 values fit in FP64)
        fd, gd = _device_copy(torch, f, dtype), _device_copy(torch, g, dtype)
        for _ in range(2):  # two calls in a row share the static scratch
            got = lbm.nusselt_noalloc(fd.data_ptr(), gd.data_ptr(), ncell, precision, grid, q,
                                      params, stream)
            _check(got, expect)


def test_noalloc_nusselt_with_padded_planes():
    import torch

    import paper_1710_04751_gb300 as lbm

    grid = (17, 9, 11)
    ncell = grid[0] * grid[1] * grid[2]
    plane = ncell + 45  # a caller layout with padding between population planes
    sim = lbm.LBM(grid, 15, Ra=3e3, precision=lbm.FP32)
    sim.step(120)
    expect = sim.nusselt()
    f, g = sim.get_populations()
    fp = np.zeros((15, plane), dtype=np.float32)
    gp = np.zeros((15, plane), dtype=np.float32)
    fp[:, :ncell] = f.reshape(15, ncell)
    gp[:, :ncell] = g.reshape(15, ncell)
    fd = torch.from_numpy(fp).cuda()
    gd = torch.from_numpy(gp).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        got = lbm.nusselt_noalloc(fd.data_ptr(), gd.data_ptr(), plane, lbm.FP32, grid, 15,
                                  sim.params_struct(), stream)
        _check(got, expect)
