"""Form B of the oracle: the cascaded collisions restated as their plain definition.

TEST INFRASTRUCTURE.  The paper derives each cascade (Sec. 2.2 for the scalar, Appendix
A for the flow, Appendix C for D3Q7) by asking that every non-conserved central moment
relax toward its equilibrium at its own rate.  This module writes that definition out
directly with linear algebra, independently of the closed forms in lbm_oracle.c:

  1. central moments kappa_b = sum_a p_a P_b(e_a - u) for the chosen combinations P_b
     (the central-moment counterpart of the basis K_b, Sec. 2.2: 0; x, y, z; xy, xz, yz;
     xx-yy; xx+yy-2zz; xx+yy+zz; xyy; xxy; xxz; xyz; xxyy -- for D3Q7 the first seven
     with the three second-order combinations xx-yy, xx+yy-2zz, xx+yy+zz);
  2. relaxation kappa~_b = kappa_b + omega_b (kappa^eq_b - kappa_b) (Eq. 15 for the scalar
     equilibria; Maxwellian equilibria with c_s^2 = 1/3 for the flow);
  3. post-collision populations solve  C(u) p~ = kappa~  (C the 15x15 or 7x7 matrix of
     step 1).

It is used only to check the closed forms ("Form A"): a wrong sign, index or term in
either form shows up as a mismatch.
"""
import numpy as np

CS2 = 1.0 / 3.0

E15 = np.array([
    [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1],
    [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1],
    [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1],
], dtype=np.float64).T  # (15, 3), the velocity list of Sec. 2.2
E7 = E15[:7]


def central_matrix(u, q=15):
    """Rows: the central-moment combinations of step 1, evaluated at e_a - u."""
    e = (E15 if q == 15 else E7) - np.asarray(u, dtype=np.float64)[None, :]
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    one = np.ones_like(x)
    if q == 7:
        rows = [one, x, y, z, x * x - y * y, x * x + y * y - 2 * z * z, x * x + y * y + z * z]
    else:
        rows = [one, x, y, z, x * y, x * z, y * z,
                x * x - y * y, x * x + y * y - 2 * z * z, x * x + y * y + z * z,
                x * y * y, x * x * y, x * x * z, x * y * z, x * x * y * y]
    return np.array(rows)


def _second_order(k7, k8, k9):
    """Individual xx, yy from the combinations xx-yy, xx+yy-2zz, xx+yy+zz."""
    zz = (k9 - k8) / 3.0
    s = k9 - zz  # xx + yy
    return 0.5 * (s + k7), 0.5 * (s - k7)


def thermal_collide(gbar, u, omega, cs2_phi=CS2, R=0.0):
    """Scalar collision with source R (Sec. 2.2, App. C; Eqs. 12-16, 25).  The source's
    only non-zero central moment is the zeroth, R.  phi = sum gbar + R/2.  The zeroth
    moment gains R; the first-order moments of gbar relax toward 0; every higher moment
    of (gbar + S) -- equal to gbar's, since S has no higher central moments -- relaxes
    toward its equilibrium at phi."""
    gbar = np.asarray(gbar, dtype=np.float64)
    q = gbar.shape[0]
    C = central_matrix(u, q)
    kap = C @ gbar
    phi = kap[0] + 0.5 * R
    eq = np.zeros(q)
    if q == 15:
        eq[9] = 3.0 * cs2_phi * phi          # xx + yy + zz -> 3 c_sphi^2 phi
        eq[14] = cs2_phi * cs2_phi * phi     # xxyy -> c_sphi^4 phi
    else:
        eq[6] = 3.0 * cs2_phi * phi
    om = np.asarray(omega, dtype=np.float64)[:q]
    post = kap + om * (eq - kap)
    post[0] = kap[0] + R
    return np.linalg.solve(C, post)


def scalar_source(q, R, u):
    """S whose central moments (the q combinations) are R for the zeroth, 0 otherwise."""
    G = np.zeros(q)
    G[0] = R
    return np.linalg.solve(central_matrix(u, q), G)


def source_central_moments(F):
    """Reading R2: central moments of the Maxwellian forcing term F.(xi-u)/(rho cs^2) f^M
    for the 15 combinations: first order F, xyy/xxy/xxz = cs^2 F, all others 0."""
    Fx, Fy, Fz = map(float, F)
    G = np.zeros(15)
    G[1], G[2], G[3] = Fx, Fy, Fz
    G[10], G[11], G[12] = CS2 * Fx, CS2 * Fy, CS2 * Fz
    return G


def flow_source(F, u):
    """S with the central moments of source_central_moments(F) about u."""
    return np.linalg.solve(central_matrix(u, 15), source_central_moments(F))


def flow_collide(fbar, F, omega, e4_mode=0):
    """Flow collision with forcing (Appendix A, defined as a central-moment relaxation):
    u from Eq. (3); the moments that relax are those of (fbar + S) about u; mass and
    momentum are not relaxed; post-collision populations are the solution of
    C(u) f~ = kappa~.  Returns (f~, rho, u)."""
    fbar = np.asarray(fbar, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    rho = fbar.sum()
    u = (E15.T @ fbar + 0.5 * F) / rho
    C = central_matrix(u, 15)
    S = np.linalg.solve(C, source_central_moments(F))
    kap = C @ (fbar + S)
    om = np.asarray(omega, dtype=np.float64).copy()
    om[:4] = 0.0
    eq = np.zeros(15)
    eq[0] = rho
    eq[9] = 3.0 * CS2 * rho          # xx + yy + zz -> 3 c_s^2 rho
    post = kap.copy()
    post[4:10] = kap[4:10] + om[4:10] * (eq[4:10] - kap[4:10])
    post[10:14] = kap[10:14] + om[10:14] * (eq[10:14] - kap[10:14])
    if e4_mode == 1:
        E = rho * CS2 * CS2
    else:
        kxx, kyy = _second_order(post[7], post[8], post[9])
        E = kxx * kyy / rho
    post[14] = kap[14] + om[14] * (E - kap[14])
    return np.linalg.solve(C, post), rho, u


def flow_equilibrium(rho, u):
    """Populations whose central moments are the flow equilibria (Maxwellian, cs^2 = 1/3)."""
    eq = np.zeros(15)
    eq[0] = rho
    eq[9] = 3.0 * CS2 * rho
    eq[14] = CS2 * CS2 * rho
    return np.linalg.solve(central_matrix(u, 15), eq)


def thermal_equilibrium(phi, u, q=15, cs2_phi=CS2):
    """Populations whose central moments are the scalar equilibria of Eq. (15)."""
    eq = np.zeros(q)
    eq[0] = phi
    if q == 15:
        eq[9] = 3.0 * cs2_phi * phi
        eq[14] = cs2_phi * cs2_phi * phi
    else:
        eq[6] = 3.0 * cs2_phi * phi
    return np.linalg.solve(central_matrix(u, q), eq)
