"""The z-slab decomposition (include/lbm_slabs.h) against one context on the whole grid,
bit for bit in every storage precision (the slabs run the same per-node code and the
halo planes hold exact copies), and its FP64 form against the oracle."""
import math

import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import params_of, random_state

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12


def lbm_mod():
    import paper_1710_04751_gb300 as lbm
    return lbm


def _pair(p, precision, nslabs, owned=None, residual_interval=50):
    lbm = lbm_mod()
    from paper_1710_04751_gb300 import slabs
    grid = (p.nx, p.ny, p.nz)
    one = lbm.LBM(grid, p.q_g, params=params_of(p), precision=precision,
                  residual_interval=residual_interval)
    dec = slabs.Slabs(grid, nslabs, p.q_g, params=params_of(p), owned=owned, precision=precision,
                      residual_interval=residual_interval)
    return one, dec


def _assert_same(one, dec):
    f1, g1 = one.get_populations()
    f2, g2 = dec.get_populations()
    assert np.array_equal(f1, f2), f"f differs at {np.argwhere(f1 != f2)[:3].tolist()}"
    assert np.array_equal(g1, g2), f"g differs at {np.argwhere(g1 != g2)[:3].tolist()}"


# (grid, lattice, precision name, nslabs, owned): even nx takes the two-node kernel in the
# 16-bit forms, odd nx the one-node kernel; uneven splits, one plane per slab, one slab;
# plane sizes that take the exchange's 16-, 4- and 2-byte copies
CASES = [
    ((12, 10, 17), 15, "FP64", 3, None),
    ((20, 12, 23), 15, "FP32", 2, [5, 18]),
    ((20, 12, 23), 7, "FP32", 4, None),
    ((20, 12, 23), 15, "FP16_DEV", 3, [1, 11, 11]),
    ((20, 12, 23), 7, "BF16_DEV", 2, None),
    ((21, 12, 23), 15, "FP16_DEV", 2, None),
    ((16, 8, 6), 15, "FP32", 6, None),
    ((16, 8, 9), 15, "FP32", 1, None),
    ((21, 11, 13), 7, "BF16_DEV", 3, None),  # odd nx*ny: 462-byte planes, 2-byte copies
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0][0]}x{c[0][1]}x{c[0][2]}-q{c[1]}-{c[2]}-s{c[3]}" for c in CASES])
def test_slabs_follow_one_context_bitwise(case):
    lbm = lbm_mod()
    grid, q, prec, nslabs, owned = case
    p = oracle.Problem.cavity(grid[0], 1e5, q_g=q, ny=grid[1], nz=grid[2])
    one, dec = _pair(p, getattr(lbm, prec), nslabs, owned)
    # the seeded initial state: every slab draws the noise of its nodes' global indices
    _assert_same(one, dec)
    # 121 steps from a random state: single steps up to the first residual check at 50,
    # then a graph of 50 steps, then single steps again
    F, G = random_state(p, 11 + grid[2])
    one.set_populations(F, G)
    dec.set_populations(F, G)
    for n in (1, 49, 50, 21):
        one.step(n)
        dec.step(n)
    assert dec.steps_done == one.steps_done == 121
    _assert_same(one, dec)
    assert dec.residual() == one.residual() > 0
    a, b = one.fields(), dec.fields()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    one.close()
    dec.close()


@pytest.mark.parametrize("bc,nslabs", [(6, 2), (6, 3), (7, 4)])
def test_slabs_periodic_z_wrap(bc, nslabs):
    # periodic z: the first and last slab exchange across the wrap as well
    lbm = lbm_mod()
    p = oracle.Problem(12, 10, 11, q_g=15, boundary=bc, omega_nu=1.7, omega_phi=1.6, gbeta=2e-3,
                       T_hot=0.6, T_cold=-0.4, U0=0.05,
                       ext_force=(1e-4, -2e-4, 5e-5) if bc == oracle.BC_PERIODIC else (0, 0, 0))
    for prec in (lbm.FP64, lbm.FP32):
        one, dec = _pair(p, prec, nslabs, residual_interval=10)
        F, G = random_state(p, 7)
        one.set_populations(F, G)
        dec.set_populations(F, G)
        one.step(23)
        dec.step(23)
        _assert_same(one, dec)
        if prec == lbm.FP64:
            F, G = p.run(F, G, 23)
            f, g = dec.get_populations()
            assert np.abs(f - F).max() <= FP64_TOL and np.abs(g - G).max() <= FP64_TOL
        one.close()
        dec.close()


@pytest.mark.parametrize("q", [15, 7])
def test_slabs_fp64_against_oracle(q):
    lbm = lbm_mod()
    from paper_1710_04751_gb300 import slabs
    p = oracle.Problem.cavity(10, 1e4, q_g=q, ny=8, nz=9)
    dec = slabs.Slabs((10, 8, 9), 3, q, params=params_of(p), precision=lbm.FP64, owned=[2, 4, 3])
    F, G = random_state(p, 3)
    dec.set_populations(F, G)
    for n in (1, 6):
        dec.step(n)
        F, G = p.run(F, G, n)
        f, g = dec.get_populations()
        assert np.abs(f - F).max() <= FP64_TOL and np.abs(g - G).max() <= FP64_TOL
    fl, fr = dec.fields(), p.fields(F, G)
    for k in fl:
        assert np.abs(fl[k] - fr[k]).max() <= 1e-12, k
    dec.close()


def test_slabs_halo_bytes_and_plan():
    lbm = lbm_mod()
    from paper_1710_04751_gb300 import slabs
    p = oracle.Problem.cavity(16, 1e4, ny=8, nz=12)
    for prec, rs, extra in ((lbm.FP32, 4, 0), (lbm.FP16_DEV, 2, 4), (lbm.FP64, 8, 0)):
        dec = slabs.Slabs((16, 8, 12), 3, 15, params=params_of(p), precision=prec)
        # two cuts, each copied both ways: 30 population planes (+ FP32 node temperatures)
        assert dec.halo_bytes == 2 * 2 * 16 * 8 * (30 * rs + extra)
        assert dec.count == 3
        assert dec.plan == {"z0": [0, 4, 8], "nz_owned": [4, 4, 4], "halo_lo": [0, 1, 1],
                            "halo_hi": [1, 1, 0]}
        dec.close()


def test_slabs_seeded_state_matches_at_128():
    # the bench's grid: two slabs of 128^3 at Ra = 1e5, 200 steps (four graphs of 50)
    lbm = lbm_mod()
    p = oracle.Problem.cavity(128, 1e5)
    one, dec = _pair(p, lbm.FP32, 2)
    one.step(200)
    dec.step(200)
    _assert_same(one, dec)
    assert dec.residual() == one.residual()
    one.close()
    dec.close()
