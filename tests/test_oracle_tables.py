"""Pins of the oracle's lattice tables against what the paper prints (CPU only)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import formb
from tests.golden_io import GOLDEN, int_rows

NORMS15 = [15, 10, 10, 10, 8, 8, 8, 4, 12, 18, 160, 160, 160, 8, 1440]


def test_velocity_set_is_the_papers():
    # Sec. 2.2: the components |e_x>, |e_y>, |e_z> of the D3Q15 lattice
    e = oracle.velocities(15)
    assert e[:, 0].tolist() == [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1]
    assert e[:, 1].tolist() == [0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1]
    assert e[:, 2].tolist() == [0, 0, 0, 0, 0, 1, -1, 1, 1, 1, 1, -1, -1, -1, -1]
    assert np.array_equal(oracle.velocities(7), e[:7])  # App. C: D3Q7 is the subset


def test_opposites():
    e = oracle.velocities(15)
    opp = oracle.opposite(15)
    for a in range(15):
        assert np.array_equal(e[opp[a]], -e[a])
    assert opp.tolist() == [0, 2, 1, 4, 3, 6, 5, 14, 13, 12, 11, 10, 9, 8, 7]


def test_k15_matches_printed_backtransform():
    rows = int_rows("backtransform_d3q15.txt")
    K = oracle.kmatrix(15)  # K[b, a]
    for a in range(15):
        assert rows[str(a)] == K[:, a].tolist(), f"row alpha={a}"


def test_k7_matches_printed_backtransform():
    rows = int_rows("backtransform_d3q7.txt")
    K = oracle.kmatrix(7)
    for a in range(7):
        assert rows[str(a)] == K[:, a].tolist(), f"row alpha={a}"


def test_k15_orthogonal_with_norms():
    K = oracle.kmatrix(15)
    G = K @ K.T
    assert np.array_equal(G, np.diag(NORMS15))


def test_k7_orthogonal():
    K = oracle.kmatrix(7)
    assert np.array_equal(K @ K.T, np.diag([7, 2, 2, 2, 4, 12, 42]))


def _gram_schmidt(T):
    out = []
    for t in T:
        v = t.astype(np.float64).copy()
        for o in out:
            v -= (v @ o) / (o @ o) * o
        out.append(v)
    return np.array(out)


def test_k15_is_gram_schmidt_of_monomial_basis():
    # Sec. 2.2: K is Gram-Schmidt applied to T_0..T_14 in order
    e = oracle.velocities(15).astype(np.float64)
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    e2 = x * x + y * y + z * z
    T = np.array([np.ones(15), x, y, z, x * y, x * z, y * z, x * x - y * y, x * x - z * z, e2,
                  x * e2, y * e2, z * e2, x * y * z,
                  x * x * y * y + x * x * z * z + y * y * z * z])
    GS = _gram_schmidt(T)
    K = oracle.kmatrix(15).astype(np.float64)
    for b in range(15):
        # parallel: |<K,GS>| = |K| |GS|
        c = K[b] @ GS[b]
        assert abs(abs(c) - np.linalg.norm(K[b]) * np.linalg.norm(GS[b])) < 1e-9, b


def test_k7_is_gram_schmidt_of_monomial_basis():
    e = oracle.velocities(7).astype(np.float64)
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    T = np.array([np.ones(7), x, y, z, x * x - y * y, x * x - z * z, x * x + y * y + z * z])
    GS = _gram_schmidt(T)
    K = oracle.kmatrix(7).astype(np.float64)
    for b in range(7):
        c = K[b] @ GS[b]
        assert abs(abs(c) - np.linalg.norm(K[b]) * np.linalg.norm(GS[b])) < 1e-9, b


def _kinv_fraction(K):
    q = K.shape[0]
    norms = [int((K[b] * K[b]).sum()) for b in range(q)]
    return [[Fraction(int(K[b, a]), norms[b]) for b in range(q)] for a in range(q)]


def test_appendix_b_source_inversion():
    rows = int_rows("source_inverse_d3q15.txt")
    inv = _kinv_fraction(oracle.kmatrix(15))
    for a in range(15):
        den, *coef = rows[str(a)]
        assert [Fraction(c, den) for c in coef] == inv[a], f"S_{a}"


def test_appendix_c_source_inversion_with_typo_reading():
    rows = int_rows("source_inverse_d3q7.txt")
    inv = _kinv_fraction(oracle.kmatrix(7))
    for a in range(7):
        den, *coef = rows[str(a)]
        if a in (3, 4):
            # printed with m^_1 for m^_2 (reading R14); moving the coefficient fixes it
            coef[2], coef[1] = coef[1], 0
        assert [Fraction(c, den) for c in coef] == inv[a], f"S_{a}"


def test_raw_moments_of_k_h():
    # Sec. 2.2: raw moments of (K . h^) as linear combinations of h^_1..h^_14
    e = oracle.velocities(15)
    K = oracle.kmatrix(15)
    rows = {}
    for line in open(GOLDEN + "/kh_raw_moments_d3q15.txt"):
        line = line.split("#", 1)[0].strip()
        if line:
            mnp, coef = line.split(":")
            rows[tuple(int(v) for v in mnp.split())] = [int(v) for v in coef.split()]
    assert len(rows) == 20
    for (m, n, p), coef in rows.items():
        mono = e[:, 0] ** m * e[:, 1] ** n * e[:, 2] ** p
        got = (K * mono[None, :]).sum(axis=1)  # coefficient of h^_b
        assert got[1:].tolist() == coef[1:], (m, n, p)


@pytest.mark.parametrize("cs2", [1.0 / 3.0, 0.25])
def test_rest_weights_reproduce_equilibrium_moments(cs2):
    e = oracle.velocities(15).astype(np.float64)
    x, y, z = e[:, 0], e[:, 1], e[:, 2]
    for q in (15, 7):
        w = oracle.weights_thermal(q, cs2)
        xs, ys, zs = x[:q], y[:q], z[:q]
        assert abs(w.sum() - 1.0) < 1e-15
        for comp in (xs, ys, zs):
            assert abs(w @ comp) < 1e-15
            assert abs(w @ (comp * comp) - cs2) < 1e-15  # Eq. 15: kappa_xx^eq = cs^2 phi
        assert abs(w @ (xs * ys)) < 1e-15
        if q == 15:
            assert abs(w @ (xs * xs * ys * ys) - cs2 * cs2) < 1e-15  # kappa_xxyy^eq
        np.testing.assert_allclose(w, formb.thermal_equilibrium(1.0, [0, 0, 0], q, cs2),
                                   atol=1e-15)
    assert np.allclose(oracle.weights_thermal(15, 1 / 3), [2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
    if cs2 == 1.0 / 3.0:
        assert np.allclose(oracle.weights_thermal(7, cs2), [0.0] + [1 / 6] * 6)
    else:
        assert np.allclose(oracle.weights_thermal(7, cs2), [0.25] + [0.125] * 6)


def test_flow_weights():
    w = oracle.weights_flow()
    np.testing.assert_allclose(w, [2 / 9] + [1 / 9] * 6 + [1 / 72] * 8, atol=1e-16)
    np.testing.assert_allclose(w, formb.flow_equilibrium(1.0, [0, 0, 0]), atol=1e-15)


def test_splitmix64_published_sequence():
    # splitmix64 seeded with 0: the published first two outputs
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
