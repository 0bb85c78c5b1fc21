"""The batched form (include/lbm_batch.h) on the GPU: every member against the FP64
oracle, the three launch modes and every tiling against each other, the batch against
single-cavity contexts, convergence and divergence handling, the autotuner, and the
64-cavity sweep at full size on sampled members.

Tolerances: FP64 max-abs 1e-12 against the oracle; FP32 the relative bound of
test_gpu_parity (1e-5 of max(|p|, weight)); equalities between launch modes, tilings and
the single-cavity kernel are bitwise (the same per-node code runs in every case).
"""
import math

import numpy as np
import pytest

import oracle
from tests import inputs
from tests.test_gpu_parity import FP64_TOL, assert_fp32_close, params_of, random_state

pytestmark = pytest.mark.gpu


def lbm_mod():
    import paper_1710_04751_gb300 as lbm
    return lbm


def member_problems(q, seed):
    """Uneven members: ragged cavities, both adiabatic forms, a periodic box with a body
    force, a heat source; random rates."""
    shapes = [
        (13, 7, 5, oracle.BC_CAVITY, 1, 0, 0.0),
        (9, 11, 6, oracle.BC_CAVITY, 0, 1, 0.0),
        (33, 5, 4, oracle.BC_PERIODIC, 1, 0, 0.0),
        (6, 9, 10, oracle.BC_ADIABATIC_BOX, 1, 0, 2e-3),
        (20, 3, 3, oracle.BC_CAVITY, 1, 0, 0.0),
    ]
    out = []
    for n, (nx, ny, nz, bc, am, e4, R) in enumerate(shapes):
        s = seed + 17 * n
        om_f = [1.0] * 4 + list(inputs.random_rates(11, s, 0.6, 1.95))
        om_g = [1.0] + list(inputs.random_rates(q - 1, s + 1, 0.6, 1.95)) + [1.0] * (15 - q)
        out.append(oracle.Problem(nx, ny, nz, q_g=q, boundary=bc, adiabatic_mode=am, e4_mode=e4,
                                  omega_f=om_f, omega_g=om_g, gbeta=2e-3, T_hot=0.6, T_cold=-0.4,
                                  ext_force=(1e-4, -2e-4, 5e-5) if bc == oracle.BC_PERIODIC else (0, 0, 0),
                                  U0=0.05, heat_source=R))
    return out


def make_batch(problems, precision, **kw):
    lbm = lbm_mod()
    members = [{"grid": (p.nx, p.ny, p.nz), "params": params_of(p)} for p in problems]
    return lbm.Batch(members, lattice=problems[0].q_g, precision=precision, **kw)


@pytest.mark.parametrize("q", [15, 7])
@pytest.mark.parametrize("mode", ["graph", "launch", "sequential"])
def test_fp64_members_match_oracle(q, mode):
    lbm = lbm_mod()
    probs = member_problems(q, 40 + q)
    b = make_batch(probs, lbm.FP64, residual_interval=4)
    states = []
    for i, p in enumerate(probs):
        F, G = random_state(p, 70 + i)
        b.member(i).set_populations(F, G)
        states.append((F, G))
    for n in (1, 3, 8):  # crosses residual checks; 8 = two whole graphs in graph mode
        b.step(n, mode=mode)
        for i, p in enumerate(probs):
            F, G = p.run(*states[i], n)
            states[i] = (F, G)
            f, g = b.member(i).get_populations()
            assert np.abs(f - F).max() <= FP64_TOL, (i, n)
            assert np.abs(g - G).max() <= FP64_TOL, (i, n)
    st = b.status()
    assert all(s["state"] == "active" and s["steps"] == 12 for s in st)
    # the residual of the last check (steps 8 -> 12) is max |dT| of each member
    for i, p in enumerate(probs):
        assert st[i]["residual"] >= 0
    b.close()


def test_fp64_residual_is_max_temperature_change_per_member():
    lbm = lbm_mod()
    probs = member_problems(15, 90)
    b = make_batch(probs, lbm.FP64, residual_interval=6)
    starts = []
    for i, p in enumerate(probs):
        F, G = random_state(p, 11 + i)
        b.member(i).set_populations(F, G)
        starts.append((F, G))
    b.step(6)
    st = b.status()
    for i, p in enumerate(probs):
        F6, G6 = p.run(*starts[i], 6)
        expect = np.abs(p.fields(F6, G6)["T"] - p.fields(*starts[i])["T"]).max()
        assert st[i]["residual"] == pytest.approx(expect, rel=1e-9), i
    b.close()


@pytest.mark.parametrize("q", [15, 7])
def test_fp32_one_step_against_oracle(q):
    lbm = lbm_mod()
    probs = member_problems(q, 120 + q)
    b = make_batch(probs, lbm.FP32, residual_interval=2)
    starts = []
    for i, p in enumerate(probs):
        F, G = random_state(p, 5 + i)
        m = b.member(i)
        m.set_populations(F, G)
        starts.append(m.get_populations())  # the FP32-rounded state both sides start from
    b.step(1)
    for i, p in enumerate(probs):
        F1, G1 = p.step(*starts[i])
        f1, g1 = b.member(i).get_populations()
        assert_fp32_close(p, f1, g1, F1, G1)
    b.close()


def test_modes_and_tilings_are_bitwise_equal():
    lbm = lbm_mod()
    members = [{"grid": (n, n, n), "Ra": Ra, "Pr": Pr}
               for n, Ra, Pr in [(24, 1e4, 0.71), (17, 3e3, 7.0), (32, 1e5, 1.0), (9, 1e3, 0.71)]]
    ref = lbm.Batch(members, precision=lbm.FP32, residual_interval=10, autotune_steps=0)
    trials = ref.autotune(trial_steps=1)
    ref.step(30, mode="sequential")
    want = [ref.member(i).get_populations() for i in range(len(members))]
    for t in trials:
        for mode in ("graph", "launch"):
            tiling = {k: t[k] for k in ("threads", "min_blocks", "mapping", "blocks_per_sm", "tile_factor")}
            b = lbm.Batch(members, precision=lbm.FP32, residual_interval=10, tiling=tiling)
            assert b.tiling == tiling
            b.step(30, mode=mode)
            for i in range(len(members)):
                f, g = b.member(i).get_populations()
                assert np.array_equal(f, want[i][0]) and np.array_equal(g, want[i][1]), (tiling, mode, i)
            b.close()
    ref.close()


def test_members_equal_single_contexts():
    """A member follows the trajectory lbm_step gives the same cavity (seed + index)."""
    lbm = lbm_mod()
    members = [{"grid": (n, n, n), "Ra": Ra, "Pr": Pr}
               for n, Ra, Pr in [(20, 1e4, 0.71), (33, 2e4, 1.0), (16, 1e3, 7.0)]]
    b = lbm.Batch(members, precision=lbm.FP32, seed=7, residual_interval=50)
    b.step(150)
    for i, m in enumerate(members):
        s = lbm.LBM(m["grid"], 15, Ra=m["Ra"], Pr=m["Pr"], precision=lbm.FP32, seed=7 + i,
                    residual_interval=50)
        s.step(150)
        f, g = s.get_populations()
        fb, gb = b.member(i).get_populations()
        assert np.array_equal(f, fb) and np.array_equal(g, gb), i
        assert b.member(i).residual() == pytest.approx(s.residual(), rel=1e-6, abs=1e-12)
        s.close()
    b.close()


def test_members_stop_at_convergence():
    lbm = lbm_mod()
    members = [{"grid": (n, n, n), "Ra": 1e3, "Pr": 0.71} for n in (8, 12, 16)]
    tol = 1e-6
    b = lbm.Batch(members, precision=lbm.FP64, residual_interval=100, steady_tol=tol)
    b.step(200_000)
    st = b.status()
    assert all(s["state"] == "converged" for s in st), st
    assert all(0 <= s["residual"] < tol for s in st)
    steps = [s["steps"] for s in st]
    assert steps == sorted(steps) and steps[0] < steps[-1]  # larger cavities take longer
    assert b.steps_done == steps[-1] and b.active_nodes == 0
    # a stopped member keeps its state
    before = b.member(0).get_populations()
    b.step(1000)
    after = b.member(0).get_populations()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert b.member(0).steps_done == steps[0]
    nu = b.member(2).nusselt()
    assert nu["hot_wall_mean"] == pytest.approx(nu["cold_wall_mean"], rel=1e-6)
    b.close()


def test_diverged_member_stops_and_the_rest_go_on():
    lbm = lbm_mod()
    members = [{"grid": (n, n, n), "Ra": 1e3, "Pr": 0.71} for n in (10, 11, 12)]
    b = lbm.Batch(members, precision=lbm.FP32, residual_interval=20)
    m1 = b.member(1)
    f, g = m1.get_populations()
    g[0, 3, 4, 5] = np.nan
    m1.set_populations(f, g)
    b.step(60)
    st = b.status()
    assert [s["state"] for s in st] == ["active", "diverged", "active"]
    assert st[1]["steps"] == 20 and st[0]["steps"] == 60 and st[2]["steps"] == 60
    assert b.active_nodes == 10 ** 3 + 12 ** 3
    b.close()


def test_member_contexts_are_owned_by_the_batch():
    lbm = lbm_mod()
    b = lbm.Batch([{"grid": (8, 8, 8), "Ra": 1e3, "Pr": 0.71}], precision=lbm.FP32,
                  autotune_steps=0)
    m = b.member(0)
    with pytest.raises(lbm.LBMError):
        m.step(1)
    m.close()  # a view: the batch still owns the member
    b.step(4)
    assert b.member(0).steps_done == 4
    b.close()


def test_invalid_batches_are_rejected():
    lbm = lbm_mod()
    one = [{"grid": (8, 8, 8), "Ra": 1e3, "Pr": 0.71}]
    with pytest.raises(lbm.LBMError):
        lbm.Batch(one, precision=lbm.FP16_DEV)
    with pytest.raises(lbm.LBMError):
        lbm.Batch(one, residual_interval=7)
    with pytest.raises(lbm.LBMError):
        lbm.Batch(one, tiling={"threads": 96, "min_blocks": 1, "mapping": 0, "blocks_per_sm": 1,
                               "tile_factor": 1})
    with pytest.raises(lbm.LBMError):
        lbm.Batch(one, tiling={"threads": 128, "min_blocks": 6, "mapping": 0, "blocks_per_sm": 1,
                               "tile_factor": 3})
    b = lbm.Batch(one, autotune_steps=0)
    with pytest.raises(lbm.LBMError):
        b.set_tiling(threads=128, min_blocks=6, mapping=0, blocks_per_sm=10_000, tile_factor=1)
    b.close()


def test_autotuner_times_every_candidate_and_keeps_the_fastest():
    lbm = lbm_mod()
    members = [{"grid": (n, n, n), "Ra": 1e4, "Pr": 0.71} for n in (32, 48, 40)]
    b = lbm.Batch(members, precision=lbm.FP32, autotune_steps=0)
    f0 = [b.member(i).get_populations() for i in range(3)]
    trials = b.autotune(trial_steps=2)
    # 4 kernel builds x 2 tile shapes x 3 tile sizes x persistent / one block per tile
    assert len(trials) == 48
    assert len({(t["threads"], t["min_blocks"], t["mapping"], t["tile_factor"], t["blocks_per_sm"] > 0)
                for t in trials}) == 48
    assert all(t["ms_per_step"] > 0 for t in trials)
    best = min(trials, key=lambda t: t["ms_per_step"])
    assert b.tiling == {k: best[k] for k in ("threads", "min_blocks", "mapping", "blocks_per_sm",
                                             "tile_factor")}
    for i in range(3):  # tuning leaves the state alone
        f, g = b.member(i).get_populations()
        assert np.array_equal(f, f0[i][0]) and np.array_equal(g, f0[i][1])
    b.close()


# ------------------------------------------------------------------------------------
# The 64-cavity sweep (edge 32/48/64/96, Ra log-uniform in [1e3, 1e6], Pr in
# {0.71, 1, 7}, seed 1) at full size, FP32, autotuned, graph mode: sampled members
# against the oracle and the single-cavity kernel
# ------------------------------------------------------------------------------------

@pytest.mark.timeout(900)
def test_sweep_of_64_cavities_sampled_members():
    lbm = lbm_mod()
    from paper_1710_04751_gb300.workloads import cavity_sweep
    members = cavity_sweep(64, seed=1)
    b = lbm.Batch(members, precision=lbm.FP32, residual_interval=100)
    assert b.count == 64 and b.active_nodes == sum(m["grid"][0] ** 3 for m in members)
    small = [i for i, m in enumerate(members) if m["grid"][0] == 32][:2]
    starts = {i: b.member(i).get_populations() for i in small}
    b.step(2, mode="launch")
    for i in small:
        m = members[i]
        p = oracle.Problem.cavity(m["grid"][0], m["Ra"], Pr=m["Pr"])
        F, G = p.run(*starts[i], 2)
        f, g = b.member(i).get_populations()
        assert_fp32_close(p, f, g, F, G, factor=2.0)
    b.step(198)  # whole graphs from step 100 on
    big = [i for i, m in enumerate(members) if m["grid"][0] == 96][:1]
    for i in small[:1] + big:
        m = members[i]
        s = lbm.LBM(m["grid"], 15, Ra=m["Ra"], Pr=m["Pr"], precision=lbm.FP32, seed=1 + i)
        s.step(200)
        f, g = s.get_populations()
        fb, gb = b.member(i).get_populations()
        assert np.array_equal(f, fb) and np.array_equal(g, gb), i
        s.close()
    st = b.status()
    assert all(s["steps"] == 200 and s["residual"] >= 0 for s in st)
    b.close()
