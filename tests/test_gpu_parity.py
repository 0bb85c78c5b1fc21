"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP64 max-abs 1e-12 on every population; FP32 |d| <= 1e-5 max(|p_oracle|, w_a)
for f and 1e-5 max(|p_oracle|, w^phi_a dT) for g, the normalisation that keeps the
relative bound meaningful for populations near zero (a zero rest weight takes the
smallest non-zero weight).
"""
import math

import numpy as np
import pytest

import oracle
from tests import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_REL = 1e-5


def lbm_mod():
    import paper_1710_04751_gb300 as lbm
    return lbm


def params_of(p: "oracle.Problem"):
    return dict(omega_f=p.omega_f, omega_g=p.omega_g, gbeta=p.gbeta, T_hot=p.T_hot,
                T_cold=p.T_cold, cs2_phi=p.cs2_phi, ext_force=list(p.ext_force), U0=p.U0,
                heat_source=p.heat_source,
                e4_mode=p.e4_mode, adiabatic_mode=p.adiabatic_mode, boundary=p.boundary)


def gpu_for(p, precision, **kw):
    lbm = lbm_mod()
    return lbm.LBM((p.nx, p.ny, p.nz), p.q_g, params=params_of(p), precision=precision, **kw)


def random_state(p, seed):
    fs, gs = p.shapes()
    F = inputs.perturbed_populations(oracle.weights_flow(), fs[1:], seed, rel=0.05)
    T = inputs.uniform_field(gs[1:], seed + 1, -0.5, 0.5)
    G = oracle.weights_thermal(p.q_g, p.cs2_phi)[:, None, None, None] * T[None] + \
        inputs.perturbed_populations(np.full(p.q_g, 0.005), gs[1:], seed + 2, rel=1.0)
    return F, G


def thermal_floor(q, cs2_phi, dT):
    """w^phi_a dT, with the smallest non-zero weight standing in for a zero rest weight
    (D3Q7 at c_sphi^2 = 1/3 has w^phi_0 = 0)."""
    w = oracle.weights_thermal(q, cs2_phi)
    return np.where(w > 0, w, w[w > 0].min()) * abs(dT)


def fp32_bound(p, ref_f, ref_g):
    wf = oracle.weights_flow()[:, None, None, None]
    wg = thermal_floor(p.q_g, p.cs2_phi, p.T_hot - p.T_cold)[:, None, None, None]
    return (FP32_REL * np.maximum(np.abs(ref_f), wf), FP32_REL * np.maximum(np.abs(ref_g), wg))


def assert_fp32_close(p, got_f, got_g, ref_f, ref_g, factor=1.0):
    bf, bg = fp32_bound(p, ref_f, ref_g)
    ef = np.abs(got_f - ref_f) / bf
    eg = np.abs(got_g - ref_g) / bg
    assert ef.max() <= factor, f"f: worst {ef.max():.3g} x bound at {np.unravel_index(ef.argmax(), ef.shape)}"
    assert eg.max() <= factor, f"g: worst {eg.max():.3g} x bound at {np.unravel_index(eg.argmax(), eg.shape)}"


# ------------------------------------------------------------------------------------
# The FP64 cavity of 32^3 at Ra = 1e3, 300 steps from the seeded initial state
# ------------------------------------------------------------------------------------

def test_fp64_cavity_32_ra1e3_300_steps():
    lbm = lbm_mod()
    p = oracle.Problem.cavity(32, 1e3)
    sim = lbm.LBM((32, 32, 32), 15, Ra=1e3, Pr=0.71, Ma=0.05 * math.sqrt(3.0), precision=lbm.FP64,
                  seed=1, noise_amp=1e-6)
    F0, G0 = p.init(seed=1, noise_amp=1e-6)
    f, g = sim.get_populations()
    assert np.abs(f - F0).max() <= 1e-16 and np.abs(g - G0).max() <= 1e-16
    sim.step(300)
    F, G = p.run(F0, G0, 300)
    f, g = sim.get_populations()
    assert np.abs(f - F).max() <= FP64_TOL
    assert np.abs(g - G).max() <= FP64_TOL
    nu_ref = p.nusselt(F, G)
    nu = sim.nusselt()
    for k in ("hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_min", "umax", "wmax"):
        assert nu[k] == pytest.approx(nu_ref[k], rel=1e-10, abs=1e-12), k
    for k in ("mid_max_z", "mid_min_z", "umax_z", "wmax_x"):
        assert nu[k] == nu_ref[k], k
    assert sim.steps_done == 300
    fl = sim.fields()
    fr = p.fields(F, G)
    for k in fl:
        assert np.abs(fl[k] - fr[k]).max() <= 1e-12, k


@pytest.mark.parametrize("q", [15, 7])
def test_fp32_cavity_32_against_fp64_oracle(q):
    lbm = lbm_mod()
    p = oracle.Problem.cavity(32, 1e3, q_g=q)
    sim = lbm.LBM((32, 32, 32), q, Ra=1e3, precision=lbm.FP32)
    F0, G0 = p.init(seed=1, noise_amp=1e-6)
    f, g = sim.get_populations()
    assert_fp32_close(p, f, g, F0, G0, factor=0.1)
    # one step from the identical (FP32-rounded) state
    sim.step(1)
    F1, G1 = p.step(f, g)
    f1, g1 = sim.get_populations()
    assert_fp32_close(p, f1, g1, F1, G1)
    # 100 steps: FP32 rounding accumulates, still inside the bound
    sim.step(99)
    F, G = p.run(f, g, 100)
    f, g = sim.get_populations()
    assert_fp32_close(p, f, g, F, G)


# ------------------------------------------------------------------------------------
# Random states, random relaxation rates, every boundary mode, ragged grids
# ------------------------------------------------------------------------------------

CASES = [
    # nx, ny, nz, q, boundary, adiabatic_mode, e4_mode
    (13, 7, 5, 15, oracle.BC_CAVITY, 1, 0),
    (13, 7, 5, 7, oracle.BC_CAVITY, 1, 1),
    (9, 11, 6, 15, oracle.BC_CAVITY, 0, 0),
    (33, 17, 9, 15, oracle.BC_PERIODIC, 1, 0),
    (8, 5, 7, 7, oracle.BC_XWALLS, 1, 0),
    (6, 9, 10, 15, oracle.BC_ADIABATIC_BOX, 1, 1),
    (6, 9, 10, 15, oracle.BC_ADIABATIC_BOX, 0, 0),
    (1, 1, 1, 15, oracle.BC_CAVITY, 1, 0),
    (2, 2, 2, 7, oracle.BC_CAVITY, 1, 0),
    (1, 3, 2, 15, oracle.BC_CAVITY, 0, 1),
    (70, 3, 3, 15, oracle.BC_CAVITY, 1, 0),
]


def _case_problem(case, seed):
    nx, ny, nz, q, bc, am, e4 = case
    om_f = [1.0] * 4 + list(inputs.random_rates(11, seed, 0.6, 1.95))
    om_g = [1.0] + list(inputs.random_rates(q - 1, seed + 1, 0.6, 1.95)) + [1.0] * (15 - q)
    return oracle.Problem(nx, ny, nz, q_g=q, boundary=bc, adiabatic_mode=am, e4_mode=e4,
                          omega_f=om_f, omega_g=om_g, gbeta=2e-3, T_hot=0.6, T_cold=-0.4,
                          ext_force=(1e-4, -2e-4, 5e-5) if bc == oracle.BC_PERIODIC else (0, 0, 0),
                          U0=0.05)


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}-bc{c[4]}-am{c[5]}-e{c[6]}" for c in CASES])
def test_fp64_random_state_steps(case):
    lbm = lbm_mod()
    p = _case_problem(case, 100 + case[0] + 7 * case[2])
    F, G = random_state(p, 5 + case[1])
    sim = gpu_for(p, lbm.FP64)
    sim.set_populations(F, G)
    f, g = sim.get_populations()
    assert np.array_equal(f, F) and np.array_equal(g, G)
    for n in (1, 4):
        sim.step(n)
        F, G = p.run(F, G, n)
        f, g = sim.get_populations()
        assert np.abs(f - F).max() <= FP64_TOL and np.abs(g - G).max() <= FP64_TOL
    fl, fr = sim.fields(), p.fields(F, G)
    for k in fl:
        assert np.abs(fl[k] - fr[k]).max() <= 1e-12, k
    if p.nx >= 2:
        nu, ref = sim.nusselt(), p.nusselt(F, G)
        for k in ("hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_min", "umax", "wmax"):
            assert nu[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-11), k


@pytest.mark.parametrize("case", CASES[:6], ids=[f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}-bc{c[4]}" for c in CASES[:6]])
def test_fp32_random_state_one_step(case):
    lbm = lbm_mod()
    p = _case_problem(case, 300 + case[0])
    F, G = random_state(p, 9 + case[2])
    sim = gpu_for(p, lbm.FP32)
    sim.set_populations(F, G)
    f, g = sim.get_populations()  # the FP32-rounded state both sides start from
    sim.step(1)
    F1, G1 = p.step(f, g)
    f1, g1 = sim.get_populations()
    assert_fp32_close(p, f1, g1, F1, G1)


# ------------------------------------------------------------------------------------
# A uniform heat source R (Eq. 4; Sec. 2.2 and App. C): both lattices, every boundary
# mode, FP64 and FP32
# ------------------------------------------------------------------------------------

HEAT_CASES = [
    (13, 7, 5, 15, oracle.BC_CAVITY, 1, 0, 2e-3),
    (13, 7, 5, 7, oracle.BC_CAVITY, 0, 0, -1.5e-3),
    (33, 17, 9, 15, oracle.BC_PERIODIC, 1, 0, 4e-3),
    (8, 5, 7, 7, oracle.BC_XWALLS, 1, 1, 1e-3),
    (6, 9, 10, 15, oracle.BC_ADIABATIC_BOX, 0, 1, 3e-3),
]


def _heat_problem(case, seed):
    p = _case_problem(case[:7], seed)
    p.heat_source = case[7]
    return p


@pytest.mark.parametrize("case", HEAT_CASES, ids=[f"{c[0]}x{c[1]}x{c[2]}-q{c[3]}-bc{c[4]}-R{c[7]:g}" for c in HEAT_CASES])
def test_fp64_heat_source_steps(case):
    lbm = lbm_mod()
    p = _heat_problem(case, 500 + case[0])
    F, G = random_state(p, 21 + case[1])
    sim = gpu_for(p, lbm.FP64)
    assert sim.params()["heat_source"] == case[7]
    sim.set_populations(F, G)
    for n in (1, 5):
        sim.step(n)
        F, G = p.run(F, G, n)
        f, g = sim.get_populations()
        assert np.abs(f - F).max() <= FP64_TOL and np.abs(g - G).max() <= FP64_TOL
    fl, fr = sim.fields(), p.fields(F, G)
    for k in fl:
        assert np.abs(fl[k] - fr[k]).max() <= 1e-12, k
    nu, ref = sim.nusselt(), p.nusselt(F, G)
    for k in ("hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_min", "umax", "wmax"):
        assert nu[k] == pytest.approx(ref[k], rel=1e-9, abs=1e-11), k


@pytest.mark.parametrize("case", HEAT_CASES[:3], ids=[f"q{c[3]}-bc{c[4]}" for c in HEAT_CASES[:3]])
def test_fp32_heat_source_one_step(case):
    lbm = lbm_mod()
    p = _heat_problem(case, 700 + case[0])
    F, G = random_state(p, 31 + case[2])
    sim = gpu_for(p, lbm.FP32)
    sim.set_populations(F, G)
    f, g = sim.get_populations()
    sim.step(1)
    F1, G1 = p.step(f, g)
    f1, g1 = sim.get_populations()
    assert_fp32_close(p, f1, g1, F1, G1)


def test_heat_source_closed_box_total_scalar():
    """Adiabatic box, no flow forcing: the total scalar grows by exactly N R per step."""
    lbm = lbm_mod()
    n, R = 10, 2.5e-3
    p = oracle.Problem(n, n, n, q_g=15, boundary=oracle.BC_ADIABATIC_BOX, gbeta=0.0,
                       T_hot=0.5, T_cold=-0.5, U0=0.05, heat_source=R)
    sim = gpu_for(p, lbm.FP64, noise_amp=0.0)
    T0 = sim.fields()["T"].sum()
    sim.step(40)
    assert sim.fields()["T"].sum() - T0 == pytest.approx(40 * n ** 3 * R, rel=1e-10)


def test_non_finite_heat_source_is_rejected():
    lbm = lbm_mod()
    p = oracle.Problem.cavity(8, 1e3)
    d = params_of(p)
    d["heat_source"] = float("nan")
    with pytest.raises(lbm.LBMError):
        lbm.LBM((8, 8, 8), 15, params=d, precision=lbm.FP64)


# ------------------------------------------------------------------------------------
# Residual, divergence flag, checkpoint / restart, errors
# ------------------------------------------------------------------------------------

def test_residual_is_max_temperature_change():
    lbm = lbm_mod()
    p = oracle.Problem.cavity(12, 1e3)
    sim = lbm.LBM((12, 12, 12), 15, Ra=1e3, precision=lbm.FP64, residual_interval=10)
    assert sim.residual() < 0
    F, G = sim.get_populations()
    sim.step(25)  # checks after steps 10 and 20
    F10, G10 = p.run(F, G, 10)
    F20, G20 = p.run(F10, G10, 10)
    expect = np.abs(p.fields(F20, G20)["T"] - p.fields(F10, G10)["T"]).max()
    assert sim.residual() == pytest.approx(expect, rel=1e-9)


def test_nan_state_reports_divergence():
    lbm = lbm_mod()
    sim = lbm.LBM((8, 8, 8), 15, Ra=1e3, precision=lbm.FP32, residual_interval=5)
    f, g = sim.get_populations()
    f[3, 4, 4, 4] = np.nan
    sim.set_populations(f, g)
    with pytest.raises(lbm.LBMError) as e:
        sim.step(10)
    assert e.value.code == lbm.lbm.LBM_EDIVERGED


@pytest.mark.parametrize("precision", ["FP32", "FP64"])
def test_checkpoint_restart_is_bitwise(precision):
    lbm = lbm_mod()
    prec = getattr(lbm, precision)
    a = lbm.LBM((16, 12, 10), 7, Ra=1e4, precision=prec)
    a.step(200)
    fa, ga = a.get_populations()
    b = lbm.LBM((16, 12, 10), 7, Ra=1e4, precision=prec)
    b.step(100)
    f, g = b.get_populations()
    c = lbm.LBM((16, 12, 10), 7, Ra=1e4, precision=prec, seed=99)
    c.set_populations(f, g)
    c.step(100)
    fc, gc = c.get_populations()
    assert np.array_equal(fa, fc) and np.array_equal(ga, gc)


def test_nusselt_needs_two_nodes_across():
    lbm = lbm_mod()
    sim = lbm.LBM((1, 4, 4), 15, Ra=1e3, precision=lbm.FP32)
    with pytest.raises(lbm.LBMError) as e:
        sim.nusselt()
    assert e.value.code == lbm.lbm.LBM_EINVAL


def test_step_zero_and_negative():
    lbm = lbm_mod()
    sim = lbm.LBM((4, 4, 4), 15, Ra=1e3)
    f0, g0 = sim.get_populations()
    sim.step(0)
    f1, g1 = sim.get_populations()
    assert np.array_equal(f0, f1) and sim.steps_done == 0
    with pytest.raises(lbm.LBMError):
        sim.step(-1)


def test_library_owned_arena_and_default_stream():
    lbm = lbm_mod()
    a = lbm.LBM((10, 9, 8), 15, Ra=1e3, precision=lbm.FP64, torch_arena=False)
    b = lbm.LBM((10, 9, 8), 15, Ra=1e3, precision=lbm.FP64)
    a.step(7)
    b.step(7)
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


@pytest.mark.parametrize("precision", ["FP32", "FP64", "FP16_DEV"])
def test_checkpoint_file_restart(precision, tmp_path):
    # 200 steps straight against 100 steps, lbm_save, LBM.load (lbm_checkpoint_info +
    # lbm_create_params + lbm_restore) and 100 more: bitwise in FP32 and FP64; the 16-bit
    # form re-encodes each deviation once on restore, so it is compared through Nu
    lbm = lbm_mod()
    prec = getattr(lbm, precision)
    a = lbm.LBM((16, 12, 10), 15, Ra=1e4, precision=prec)
    a.step(200)
    b = lbm.LBM((16, 12, 10), 15, Ra=1e4, precision=prec)
    b.step(100)
    path = str(tmp_path / "state.ckpt")
    b.save(path)
    c = lbm.LBM.load(path)
    assert c.steps_done == 100 and c.precision == prec and c.params() == b.params()
    c.step(100)
    assert c.steps_done == 200
    fa, ga = a.get_populations()
    fc, gc = c.get_populations()
    if prec in (lbm.FP32, lbm.FP64):
        assert np.array_equal(fa, fc) and np.array_equal(ga, gc)
    else:
        assert c.nusselt()["hot_wall_mean"] == pytest.approx(a.nusselt()["hot_wall_mean"], rel=1e-3)
    other = lbm.LBM((16, 12, 12), 15, Ra=1e4, precision=prec)
    with pytest.raises(lbm.LBMError) as e:
        other.restore(path)
    assert e.value.code == lbm.lbm.LBM_EINVAL


@pytest.mark.parametrize("precision", ["FP32", "FP64"])
def test_native_precision_transfers(precision):
    # lbm_get/set_populations_native move the stored values themselves: round trips are
    # exact, and a step after a native upload equals a step after the FP64 upload of the
    # same values, bitwise; the 16-bit forms refuse them
    lbm = lbm_mod()
    prec = getattr(lbm, precision)
    dt = np.float32 if prec == lbm.FP32 else np.float64
    p = _case_problem((20, 9, 7, 15, oracle.BC_CAVITY, 1, 0), 77)
    F, G = random_state(p, 78)
    a = gpu_for(p, prec)
    a.set_populations(F, G)
    fn, gn = a.get_populations_native()
    assert fn.dtype == dt and np.array_equal(fn, F.astype(dt)) and np.array_equal(gn, G.astype(dt))
    b = gpu_for(p, prec)
    b.set_populations_native(fn, gn)
    fb, gb = b.get_populations()
    fa, ga = a.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.step(3)
    b.step(3)
    assert np.array_equal(a.get_populations()[0], b.get_populations()[0])
    assert np.array_equal(a.get_populations()[1], b.get_populations()[1])
    h = gpu_for(p, lbm.FP16_DEV)
    with pytest.raises(lbm.LBMError) as e:
        h.get_populations_native()
    assert e.value.code == lbm.lbm.LBM_EINVAL
