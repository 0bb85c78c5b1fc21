"""The 16-bit storage forms (FP16 / BF16 deviations from the rest state -- w_a for the flow,
w^phi_a T_node for the scalar -- with FP32 arithmetic) against the FP64 oracle and the FP32
path.

One step from a state both sides share (the GPU's own decoded state): each population
may differ from the oracle by the rounding of its stored deviation, 2^-11 |p - p_rest|
(FP16) or 2^-8 |p - p_rest| (BF16), plus the FP32 bound of the FP32 tests and, for FP16,
half the smallest subnormal step (2^-25)."""
import math

import numpy as np
import pytest

import oracle
from tests import inputs
from tests.test_gpu_parity import FP32_REL, gpu_for, random_state, thermal_floor

pytestmark = pytest.mark.gpu

EPS = {"FP16_DEV": 2.0 ** -11, "BF16_DEV": 2.0 ** -8}
SUBNORMAL_HALF = {"FP16_DEV": 2.0 ** -25, "BF16_DEV": 0.0}


def _bound(p, prec_name, ref_f, ref_g):
    wf = oracle.weights_flow()[:, None, None, None]
    # the scalar's stored deviation is from w^phi_a T of the node (T: the node's sum)
    wt = oracle.weights_thermal(p.q_g, p.cs2_phi)[:, None, None, None] * ref_g.sum(axis=0)[None]
    floor_g = thermal_floor(p.q_g, p.cs2_phi, p.T_hot - p.T_cold)[:, None, None, None]
    e, sub = EPS[prec_name], SUBNORMAL_HALF[prec_name]
    bf = e * np.abs(ref_f - wf) + FP32_REL * np.maximum(np.abs(ref_f), wf) + sub
    bg = e * np.abs(ref_g - wt) + FP32_REL * np.maximum(np.abs(ref_g), floor_g) + sub
    return bf, bg


CASES = [(13, 7, 5, 15), (9, 11, 6, 7), (32, 8, 8, 15)]


@pytest.mark.parametrize("prec_name", ["FP16_DEV", "BF16_DEV"])
@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}" for c in CASES])
def test_one_step_against_oracle(prec_name, case):
    import paper_1710_04751_gb300 as lbm
    nx, ny, nz, q = case
    p = oracle.Problem(nx, ny, nz, q_g=q, omega_nu=1.7, omega_phi=1.6, gbeta=2e-3, U0=0.05,
                       cs2_phi=1 / 3 if q == 15 else 0.25)
    F, G = random_state(p, 40 + nx)
    sim = gpu_for(p, getattr(lbm, prec_name))
    sim.set_populations(F, G)
    f, g = sim.get_populations()  # the decoded 16-bit state both sides start from
    # storing the state rounds only the deviation from the rest state
    bf0, bg0 = _bound(p, prec_name, F, G)
    assert (np.abs(f - F) <= bf0).all() and (np.abs(g - G) <= bg0).all()
    sim.step(1)
    F1, G1 = p.step(f, g)
    f1, g1 = sim.get_populations()
    bf, bg = _bound(p, prec_name, F1, G1)
    assert (np.abs(f1 - F1) <= bf).all(), np.max(np.abs(f1 - F1) / bf)
    assert (np.abs(g1 - G1) <= bg).all(), np.max(np.abs(g1 - G1) / bg)


def test_16bit_checkpoint_roundtrip():
    # the node temperature the thermal deviations refer to is rebuilt from the uploaded
    # populations, so a restore re-encodes each deviation once: within one 16-bit rounding
    import paper_1710_04751_gb300 as lbm
    for name, eps in (("FP16_DEV", 2.0 ** -11), ("BF16_DEV", 2.0 ** -8)):
        prec = getattr(lbm, name)
        a = lbm.LBM((20, 12, 10), 15, Ra=3e3, precision=prec)
        a.step(150)
        f, g = a.get_populations()
        b = lbm.LBM((20, 12, 10), 15, Ra=3e3, precision=prec, seed=5)
        b.set_populations(f, g)
        f2, g2 = b.get_populations()
        wf = oracle.weights_flow()[:, None, None, None]
        wt = oracle.weights_thermal(15)[:, None, None, None] * g.sum(axis=0)[None]
        assert np.array_equal(f, f2)  # flow offsets are constants: exact
        assert (np.abs(g2 - g) <= 2 * eps * np.abs(g - wt) + 2.0 ** -24).all()
        a.step(50)
        b.step(50)
        na, nb = a.nusselt(), b.nusselt()
        assert nb["hot_wall_mean"] == pytest.approx(na["hot_wall_mean"], rel=1e-3)


@pytest.mark.timeout(600)
def test_steady_nusselt_of_the_16bit_forms():
    # 48^3, Ra = 1e4, to max |dT| per 100 steps < 1e-6 (or 150k steps): steady Nu of FP16
    # within 0.5% of FP32; BF16 (8 significant bits) within 2%
    import paper_1710_04751_gb300 as lbm
    out = {}
    for name in ("FP32", "FP16_DEV", "BF16_DEV"):
        sim = lbm.LBM((48, 48, 48), 15, Ra=1e4, Ma=0.05 * math.sqrt(3.0),
                      precision=getattr(lbm, name))
        while sim.steps_done < 150_000:
            sim.step(2000)
            r = sim.residual()
            if 0 <= r < 1e-6:
                break
        out[name] = (sim.nusselt(), sim.steps_done, sim.residual())
    ref = out["FP32"][0]
    print({k: (v[0]["mid_mean"], v[0]["hot_wall_mean"], v[1], v[2]) for k, v in out.items()})
    for k in ("mid_mean", "hot_wall_mean"):
        assert out["FP16_DEV"][0][k] == pytest.approx(ref[k], rel=5e-3), k
        assert out["BF16_DEV"][0][k] == pytest.approx(ref[k], rel=2e-2), k
