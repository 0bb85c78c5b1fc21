"""The update at the paper's own higher-order rates (collide_unit.cuh) against the FP64
oracle, which runs the paper's closed-form cascades.  The paper relaxes every moment
whose rate it does not tie to a transport coefficient at rate 1 (Sec. 2.2, App. A, C);
the library then computes the post-collision state from the low-order moments alone.
The rates that stay free -- the five shear rates of the flow and the three first-order
rates of the scalar -- are drawn at random (all different), with random states, body
forces, heat sources, both fourth-order equilibria (R1), both adiabatic rules, every
boundary mode, ragged and degenerate grids; FP64 to 1e-12, FP32 and the 16-bit forms
(two-node pair kernel at even nx) within the bounds of test_gpu_parity.py and
test_gpu_precision.py."""
import numpy as np
import pytest

import oracle
from tests import inputs
from tests.test_gpu_parity import FP64_TOL, assert_fp32_close, gpu_for, random_state

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, nz, q, boundary, adiabatic_mode, e4_mode, heat source R, body force
    (13, 7, 5, 15, oracle.BC_CAVITY, 1, 0, 0.0, False),
    (13, 7, 5, 7, oracle.BC_CAVITY, 1, 1, 2e-3, True),
    (9, 11, 6, 15, oracle.BC_CAVITY, 0, 1, -1e-3, False),
    (33, 17, 9, 15, oracle.BC_PERIODIC, 1, 0, 3e-3, True),
    (8, 5, 7, 7, oracle.BC_XWALLS, 1, 0, 0.0, True),
    (6, 9, 10, 15, oracle.BC_ADIABATIC_BOX, 1, 1, 1e-3, False),
    (6, 9, 10, 7, oracle.BC_ADIABATIC_BOX, 0, 0, 0.0, False),
    (1, 1, 1, 15, oracle.BC_CAVITY, 1, 0, 0.0, False),
    (2, 2, 2, 7, oracle.BC_CAVITY, 1, 0, 0.0, True),
    (1, 3, 2, 15, oracle.BC_CAVITY, 0, 1, 0.0, False),
    (70, 3, 3, 15, oracle.BC_CAVITY, 1, 0, 0.0, True),
    (16, 6, 5, 15, oracle.BC_CAVITY, 1, 0, 1e-3, True),   # even nx: the 16-bit pair kernel
    (24, 5, 4, 7, oracle.BC_CAVITY, 1, 1, 0.0, False),
]
IDS = [f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}-bc{c[4]}-am{c[5]}-e{c[6]}" for c in CASES]


def unit_problem(case, seed):
    nx, ny, nz, q, bc, am, e4, R, force = case
    om_f = [1.0] * 15
    om_f[4:9] = list(inputs.random_rates(5, seed, 0.6, 1.95))
    om_g = [1.0] * 15
    om_g[1:4] = list(inputs.random_rates(3, seed + 1, 0.6, 1.95))
    p = oracle.Problem(nx, ny, nz, q_g=q, boundary=bc, adiabatic_mode=am, e4_mode=e4,
                       omega_f=om_f, omega_g=om_g, gbeta=2e-3, T_hot=0.6, T_cold=-0.4,
                       cs2_phi=1 / 3 if q == 15 else 0.25, U0=0.05,
                       ext_force=(1e-4, -2e-4, 5e-5) if force else (0, 0, 0), heat_source=R)
    return p


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp64_unit_rates_steps(case):
    import paper_1710_04751_gb300 as lbm
    p = unit_problem(case, 40 + case[0] + case[2])
    F, G = random_state(p, 3 + case[1])
    sim = gpu_for(p, lbm.FP64)
    sim.set_populations(F, G)
    for n in (1, 4):
        sim.step(n)
        F, G = p.run(F, G, n)
        f, g = sim.get_populations()
        assert np.abs(f - F).max() <= FP64_TOL, np.abs(f - F).max()
        assert np.abs(g - G).max() <= FP64_TOL, np.abs(g - G).max()


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_fp32_unit_rates_one_step(case):
    import paper_1710_04751_gb300 as lbm
    p = unit_problem(case, 60 + case[0])
    F, G = random_state(p, 8 + case[2])
    sim = gpu_for(p, lbm.FP32)
    sim.set_populations(F, G)
    f, g = sim.get_populations()
    sim.step(1)
    F1, G1 = p.step(f, g)
    f1, g1 = sim.get_populations()
    assert_fp32_close(p, f1, g1, F1, G1)


@pytest.mark.parametrize("prec_name", ["FP16_DEV", "BF16_DEV"])
@pytest.mark.parametrize("case", [c for c in CASES if c[4] == oracle.BC_CAVITY],
                         ids=[i for c, i in zip(CASES, IDS) if c[4] == oracle.BC_CAVITY])
def test_16bit_unit_rates_two_steps(prec_name, case):
    import paper_1710_04751_gb300 as lbm
    from tests.test_gpu_precision import _bound
    p = unit_problem(case, 80 + case[1])
    F, G = random_state(p, 12 + case[0])
    sim = gpu_for(p, getattr(lbm, prec_name))
    sim.set_populations(F, G)
    f, g = sim.get_populations()
    for _ in range(2):  # each step from the GPU's own decoded state
        sim.step(1)
        F1, G1 = p.step(f, g)
        f, g = sim.get_populations()
        bf, bg = _bound(p, prec_name, F1, G1)
        assert (np.abs(f - F1) <= bf).all(), np.max(np.abs(f - F1) / bf)
        assert (np.abs(g - G1) <= bg).all(), np.max(np.abs(g - G1) / bg)
