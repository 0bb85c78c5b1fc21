"""Pins of the oracle's one-cell collisions (CPU only).

Form A (the paper's closed-form cascades, lbm_oracle.c) must equal Form B (the plain
definition: relax each central moment toward its equilibrium, oracle/formb.py) for
random states and random, all-different relaxation rates, so that a dropped term, a
wrong sign or a swapped index in either form shows up.
"""
import numpy as np
import pytest

import oracle
from oracle import formb
from tests import inputs

TOL = 1e-13


def _states(n, seed):
    w = oracle.weights_flow()
    f = inputs.perturbed_populations(w, (n,), seed, rel=0.3, absolute=0.01).T
    F = inputs.random_vectors(n, seed + 1, 0.02)
    om = np.stack([inputs.random_rates(15, seed + 2 + i) for i in range(n)])
    return f, F, om


@pytest.mark.parametrize("e4_mode", [0, 1])
def test_flow_form_a_equals_form_b(e4_mode):
    f, F, om = _states(2500, 11)
    worst = 0.0
    for i in range(len(f)):
        a, rho_a, u_a = oracle.collide_flow(f[i], F[i], om[i], e4_mode)
        b, rho_b, u_b = formb.flow_collide(f[i], F[i], om[i], e4_mode)
        worst = max(worst, np.abs(a - b).max())
        assert abs(rho_a - rho_b) < TOL and np.abs(u_a - u_b).max() < TOL
    assert worst < TOL, worst


def test_flow_source_form_a_equals_form_b_and_moments():
    F = inputs.random_vectors(200, 5, 0.05)
    U = inputs.random_vectors(200, 6, 0.1)
    e = oracle.velocities(15).astype(np.float64)
    for Fi, ui in zip(F, U):
        Sa = oracle.flow_source(Fi, ui)
        np.testing.assert_allclose(Sa, formb.flow_source(Fi, ui), atol=1e-16, rtol=0)
        assert abs(Sa.sum()) < 1e-16               # no mass source
        np.testing.assert_allclose(e.T @ Sa, Fi, atol=1e-16, rtol=0)   # sum S e = F
        c = e - ui[None, :]
        # second-order central moments of S vanish (reading R2)
        for (p, q) in [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]:
            assert abs(Sa @ (c[:, p] * c[:, q])) < 1e-16
        assert abs(Sa @ (c[:, 0] * c[:, 1] ** 2) - Fi[0] / 3.0) < 1e-16


@pytest.mark.parametrize("q", [15, 7])
@pytest.mark.parametrize("cs2", [1.0 / 3.0, 0.25])
@pytest.mark.parametrize("R", [0.0, 3e-3])
def test_thermal_form_a_equals_form_b(q, cs2, R):
    n = 650  # with the flow test's 2 x 2500: about 1e4 random cell states in all
    rng_g = inputs.perturbed_populations(np.ones(q) * 0.05, (n,), 21, rel=1.0).T
    T = inputs.uniform_field((n,), 22, -0.5, 0.5)
    U = inputs.random_vectors(n, 23, 0.1)
    w = oracle.weights_thermal(q, cs2)
    worst = 0.0
    for i in range(n):
        g = w * T[i] + rng_g[i]
        om = inputs.random_rates(q, 100 + i)
        a = oracle.collide_thermal(g, U[i], om, cs2, R * (1 + T[i]))
        b = formb.thermal_collide(g, U[i], om, cs2, R * (1 + T[i]))
        worst = max(worst, np.abs(a - b).max())
    assert worst < TOL, worst


def test_flow_equilibrium_is_fixed_point():
    for i, (rho, u) in enumerate([(1.0, (0, 0, 0)), (1.03, (0.05, -0.02, 0.01)),
                                  (0.97, (-0.08, 0.04, 0.06))]):
        feq = formb.flow_equilibrium(rho, u)
        for e4 in (0, 1):
            out, r, uu = oracle.collide_flow(feq, [0, 0, 0], inputs.random_rates(15, i), e4)
            np.testing.assert_allclose(out, feq, atol=1e-15, rtol=0)
            np.testing.assert_allclose(uu, u, atol=1e-15)


@pytest.mark.parametrize("q", [15, 7])
def test_thermal_equilibrium_is_fixed_point(q):
    for i, (phi, u) in enumerate([(0.3, (0, 0, 0)), (-0.4, (0.05, -0.02, 0.01)),
                                  (1.0, (-0.08, 0.04, 0.06))]):
        for cs2 in (1.0 / 3.0, 0.25):
            geq = formb.thermal_equilibrium(phi, u, q, cs2)
            out = oracle.collide_thermal(geq, u, inputs.random_rates(q, 7 + i), cs2)
            np.testing.assert_allclose(out, geq, atol=1e-15, rtol=0)


def test_collision_invariants():
    f, F, om = _states(100, 31)
    e = oracle.velocities(15).astype(np.float64)
    for i in range(len(f)):
        out, rho, u = oracle.collide_flow(f[i], F[i], om[i], 0)
        assert abs(out.sum() - f[i].sum()) < 1e-15
        # Eq. 2a: collision adds the force to the momentum (sum (K g^) e = 0, sum S e = F)
        np.testing.assert_allclose(e.T @ out, e.T @ f[i] + F[i], atol=1e-15, rtol=0)
        g = inputs.perturbed_populations(np.full(15, 0.02), (1,), 500 + i, rel=1.0)[:, 0]
        for q in (15, 7):
            gq = g[:q]
            out_g = oracle.collide_thermal(gq, u, inputs.random_rates(q, 900 + i))
            assert abs(out_g.sum() - gq.sum()) < 1e-15  # h^_0 = 0: phi is invariant


def test_rates_of_one_are_the_equilibrium():
    # with every rate 1 the post-collision central moments are the equilibria, so the
    # collision returns the equilibrium of the same (rho, u) / (phi, u)
    f, F, _ = _states(20, 41)
    for i in range(len(f)):
        out, rho, u = oracle.collide_flow(f[i], [0, 0, 0], np.ones(15), 1)
        np.testing.assert_allclose(out, formb.flow_equilibrium(rho, u), atol=1e-15)
        g = oracle.weights_thermal(15) * 0.3 + 0.01 * f[i]
        out = oracle.collide_thermal(g, u, np.ones(15))
        np.testing.assert_allclose(out, formb.thermal_equilibrium(g.sum(), u), atol=1e-15)


@pytest.mark.parametrize("q", [15, 7])
def test_scalar_source(q):
    # Appendix B / C: S^phi has total R and, for the chosen central-moment combinations,
    # no moment other than the zeroth (Eq. 16); it equals the generic inversion
    e = oracle.velocities(q).astype(np.float64)
    for i, (R, u) in enumerate([(1e-3, (0.0, 0.0, 0.0)), (-2e-3, (0.05, -0.03, 0.02)),
                                (4e-3, (-0.1, 0.07, 0.09))]):
        S = oracle.scalar_source(q, R, u)
        assert abs(S.sum() - R) < 1e-18
        np.testing.assert_allclose(formb.central_matrix(u, q) @ S, [R] + [0.0] * (q - 1),
                                   atol=1e-18)
        np.testing.assert_allclose(S, formb.scalar_source(q, R, u), atol=1e-18)
        # the first raw moments are those the paper lists: sum S e = u R
        np.testing.assert_allclose(e.T @ S, np.array(u) * R, atol=1e-18)


def test_scalar_source_matches_printed_projections_to_second_order():
    # Eq. (19): the projections m^s_0..m^s_9 and m^s_13 printed by the paper are those of S
    # (m^s_10..12 and m^s_14 print continuous u^3 and three distinct u_i^2 u_j^2 terms that
    # the lattice cannot hold; the inversion uses the lattice moments, reading R14)
    K = oracle.kmatrix(15).astype(np.float64)
    R, (ux, uy, uz) = 2e-3, (0.05, -0.03, 0.02)
    m = K @ oracle.scalar_source(15, R, (ux, uy, uz))
    printed = {0: R, 1: ux * R, 2: uy * R, 3: uz * R, 4: ux * uy * R, 5: ux * uz * R,
               6: uy * uz * R, 7: (ux * ux - uy * uy) * R, 8: (ux * ux + uy * uy - 2 * uz * uz) * R,
               9: (ux * ux + uy * uy + uz * uz - 2) * R, 13: ux * uy * uz * R}
    for b, v in printed.items():
        assert abs(m[b] - v) < 1e-18, b


def test_third_order_part_of_the_flow_source_is_immaterial_at_the_papers_rates():
    # Reading R2 gives the flow source third-order central moments c_s^2 F (xyy, xxy, xxz).
    # The paper relaxes the third-order moments at rate 1 (App. A): their post-collision
    # values are then the equilibrium's whatever the source contributes, so dropping that
    # part of the reading changes nothing; at other third-order rates it does.
    from oracle import formb
    rng = np.random.default_rng(17)
    w = oracle.weights_flow()
    orig = formb.source_central_moments

    def first_order_only(F):
        G = orig(F)
        G[10:13] = 0.0
        return G

    for trial in range(40):
        f = w * (1 + 0.05 * rng.standard_normal(15))
        F = 1e-3 * rng.standard_normal(3)
        om = [1.0] * 15
        om[4:9] = rng.uniform(0.6, 1.95, 5)
        a, _, _ = formb.flow_collide(f, F, om, e4_mode=trial % 2)
        formb.source_central_moments = first_order_only
        try:
            b, _, _ = formb.flow_collide(f, F, om, e4_mode=trial % 2)
            om2 = list(om)
            om2[10:13] = [0.7, 1.3, 1.6]
            c, _, _ = formb.flow_collide(f, F, om2, e4_mode=trial % 2)
        finally:
            formb.source_central_moments = orig
        d, _, _ = formb.flow_collide(f, F, om2, e4_mode=trial % 2)
        assert np.abs(a - b).max() <= 1e-15
        assert np.abs(c - d).max() > 1e-8  # the reading is live at other rates
