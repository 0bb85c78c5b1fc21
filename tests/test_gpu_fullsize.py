"""Parity at the benchmark sizes, on every node and every population: the 128^3 cavity at
Ra = 1e5 (FP32 on both thermal lattices, and the 16-bit forms FP16 / BF16, whose even nx
takes the two-node pair kernel) and the 256^3 cavity at Ra = 1e6 (FP32 and FP16), in the
launch configurations bench.py and the precision study time.  After 300 steps from the
seeded initial state (so that the boundary layers, and every term of the collisions, are
active) the GPU takes one more step; the oracle takes the same step, on the whole grid,
from the GPU's own pre-step state.

Tolerances: FP32 |d| <= 1e-5 max(|p_oracle|, w_a) (flow) and 1e-5 max(|p_oracle|,
w^phi_a dT) (scalar), as in test_gpu_parity.py; the 16-bit forms add the rounding of the
stored deviation: under one unit in the last place, 2 x 2^-11 (FP16) or 2 x 2^-8 (BF16) of
|p - p_rest| and for FP16 the smallest subnormal step (2^-24; the flow deviations, stored
times 2^12, have a finer one) -- the bound of stochastic rounding (the flow), twice that of
rounding to nearest (the scalar)."""
import math

import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import FP32_REL, thermal_floor

pytestmark = pytest.mark.gpu

EPS = {"FP32": 0.0, "FP16_DEV": 2.0 ** -11, "BF16_DEV": 2.0 ** -8}
SUBNORMAL_HALF = {"FP32": 0.0, "FP16_DEV": 2.0 ** -25, "BF16_DEV": 0.0}


def whole_grid_check(n, q, prec_name, Ra, warm=300):
    import paper_1710_04751_gb300 as lbm
    p = oracle.Problem.cavity(n, Ra, q_g=q)
    sim = lbm.LBM((n, n, n), q, Ra=Ra, Pr=0.71, Ma=0.05 * math.sqrt(3.0),
                  precision=getattr(lbm, prec_name))
    sim.step(warm)
    f0, g0 = sim.get_populations()
    sim.step(1)
    f1, g1 = sim.get_populations()
    sim.close()
    F1, G1 = p.step(f0, g0)
    wf = oracle.weights_flow()
    wt = oracle.weights_thermal(q, p.cs2_phi)
    floor_g = thermal_floor(q, p.cs2_phi, p.T_hot - p.T_cold)
    e, sub = EPS[prec_name], SUBNORMAL_HALF[prec_name]
    Tref = G1.sum(axis=0)  # the node temperature the stored scalar deviations refer to
    worst = 0.0
    for a in range(15):  # one population plane at a time keeps the temporaries small
        ref = F1[a]
        bound = 2 * e * np.abs(ref - wf[a]) + FP32_REL * np.maximum(np.abs(ref), wf[a]) + 2 * sub
        r = np.abs(f1[a] - ref) / bound
        k = np.unravel_index(r.argmax(), r.shape)
        assert r.max() <= 1.0, ("f", a, k, r.max())
        worst = max(worst, r.max())
    for a in range(q):
        ref = G1[a]
        bound = 2 * e * np.abs(ref - wt[a] * Tref) + FP32_REL * np.maximum(np.abs(ref), floor_g[a]) + 2 * sub
        r = np.abs(g1[a] - ref) / bound
        k = np.unravel_index(r.argmax(), r.shape)
        assert r.max() <= 1.0, ("g", a, k, r.max())
        worst = max(worst, r.max())
    # what holds at any size: the closed cavity conserves mass
    assert abs(f1.sum() - f0.sum()) <= 1e-5 * f0.sum()
    print(f"{n}^3 q={q} {prec_name}: worst |GPU - oracle| / bound = {worst:.3f}")


@pytest.mark.timeout(300)
@pytest.mark.parametrize("prec_name", ["FP32", "FP16_DEV", "BF16_DEV"])
@pytest.mark.parametrize("q", [15, 7])
def test_whole_grid_one_step_at_128(q, prec_name):
    whole_grid_check(128, q, prec_name, 1e5)


@pytest.mark.timeout(600)
@pytest.mark.parametrize("prec_name", ["FP32", "FP16_DEV"])
def test_whole_grid_one_step_at_256(prec_name):
    # the precision study's cavity (256^3, Ra = 1e6) and the bench's 256^3 lines
    whole_grid_check(256, 15, prec_name, 1e6)
