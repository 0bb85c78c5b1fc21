"""The addressing of the 16-bit forms' two-node pair kernel (pair.cuh, step.cu), modelled
on the CPU: for every pair (2t, 2t+1) of every row away from the y and z walls, each of
the 15 flow and Q scalar loads lands on the population the pull rule (Eqs. 2b, 13b; the
x-face rules of Sec. 3) names -- the source node's population a, or at an x face the
node's own opposite population -- inside its plane, the node-temperature loads on the node
that holds the population, the 32-bit (x-aligned links, stores) and 64-bit (temperature
pairs) accesses aligned.  No GPU: the index arithmetic is restated from the kernel."""
import pytest


def ex(a): return 1 if a == 1 else -1 if a == 2 else ((-1 if (a - 7) & 1 else 1) if a >= 7 else 0)
def ey(a): return 1 if a == 3 else -1 if a == 4 else ((-1 if ((a - 7) >> 1) & 1 else 1) if a >= 7 else 0)
def ez(a): return 1 if a == 5 else -1 if a == 6 else ((-1 if (a - 7) >> 2 else 1) if a >= 7 else 0)
def opp(a): return 0 if a == 0 else ((a + 1 if a & 1 else a - 1) if a <= 6 else 21 - a)


def pair_loads(a, c0, r, P, lo, hi):
    """Element indices (population, then node temperature) the kernel reads for link a
    and the nodes c0, c0 + 1 (r = e_y nx + e_z nxy, the row offset of the source)."""
    if ex(a) == 0:
        return [a * P + c0 - r, a * P + c0 - r + 1], [c0 - r, c0 - r + 1]
    if ex(a) > 0:
        base = a * P - r - 1
        i0 = c0 + r + 1 + (opp(a) - a) * P if lo else c0
        t0 = (c0 + r + 1 if lo else c0) - r - 1
        return [base + i0, base + c0 + 1], [t0, c0 - r]
    base = a * P - r + 1
    i1 = c0 + r + (opp(a) - a) * P if hi else c0 + 1
    t1 = (c0 + r if hi else c0 + 1) - r + 1
    return [base + c0, base + i1], [c0 - r + 1, t1]


@pytest.mark.parametrize("nx,ny,nz,q", [(2, 5, 4, 15), (4, 3, 3, 7), (10, 6, 5, 15), (66, 4, 5, 15),
                                        (130, 3, 4, 7), (64, 5, 3, 15), (16, 4, 4, 15)])
def test_pair_kernel_addressing(nx, ny, nz, q):
    ncell = nx * ny * nz
    P = (ncell + 63) // 64 * 64
    nxy = nx * ny
    pairs = 0
    for k in range(1, nz - 1):
        for j in range(1, ny - 1):
            for t in range(nx // 2):
                c0 = k * nxy + j * nx + 2 * t
                lo, hi = t == 0, 2 * t + 2 == nx
                assert c0 % 2 == 0  # 32-bit two-value and 64-bit temperature-pair accesses aligned
                for n_links, planes in ((q, q), (15, 15)):
                    for a in range(n_links):
                        r = ey(a) * nx + ez(a) * nxy
                        got, got_t = pair_loads(a, c0, r, P, lo, hi)
                        for e in range(2):
                            i = 2 * t + e
                            si = i - ex(a)
                            if 0 <= si < nx:  # the source node's population a
                                node = (k - ez(a)) * nxy + (j - ey(a)) * nx + si
                                want = a * P + node
                            else:             # through an x face: the node's own opposite population
                                node = k * nxy + j * nx + i
                                want = opp(a) * P + node
                            assert got[e] == want, (a, t, e)
                            assert got_t[e] == node, (a, t, e)
                            assert 0 <= got[e] < planes * P and 0 <= got_t[e] < P
                pairs += 1
    assert pairs == (ny - 2) * (nz - 2) * (nx // 2)


def test_division_by_invariant_integers():
    # the batched kernel divides node and row indices by nx and ny as n M >> (32 + l) with
    # l = ceil(log2 d), M = ceil(2^(32+l) / d) (batch.cu); that equals n // d for n < 2^31
    import numpy as np
    rng = np.random.default_rng(3)
    for d in list(range(1, 300)) + [511, 512, 513, 1023, 1024, 4095, 65535, 2 ** 20 + 7]:
        l = 0
        while (1 << l) < d:
            l += 1
        M = -(-(1 << (32 + l)) // d)
        ns = np.concatenate([np.arange(0, 4 * d + 3), rng.integers(0, 2 ** 31, 2000),
                             [2 ** 31 - 1, 2 ** 31 - 2, (2 ** 31 - 1) // d * d, (2 ** 31 - 1) // d * d - 1]])
        for n in ns.tolist():
            assert (n * M) >> (32 + l) == n // d, (n, d)
