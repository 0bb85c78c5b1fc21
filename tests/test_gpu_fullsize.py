"""Parity at the benchmark size: 128^3, Ra = 1e5, FP32, both thermal lattices, in the
same launch configuration bench.py times.  The oracle recomputes one step for a sample
of nodes (every corner, edge and face class plus random interior nodes) from the
GPU's own pre-step state; FP32 tolerance as in test_gpu_parity.py."""
import math

import numpy as np
import pytest

import oracle
from tests import inputs
from tests.test_gpu_parity import FP32_REL, thermal_floor

pytestmark = pytest.mark.gpu

N = 128


def sample_nodes(n, seed, count=600):
    e = [0, 1, n // 2, n - 2, n - 1]
    nodes = {(i, j, k) for i in e for j in e for k in e}
    rng = np.random.default_rng(seed)
    for _ in range(count):
        nodes.add(tuple(int(v) for v in rng.integers(0, n, 3)))
    return sorted(nodes)


@pytest.mark.parametrize("q", [15, 7])
def test_sampled_nodes_at_128(q):
    import paper_1710_04751_gb300 as lbm
    p = oracle.Problem.cavity(N, 1e5, q_g=q)
    sim = lbm.LBM((N, N, N), q, Ra=1e5, Pr=0.71, Ma=0.05 * math.sqrt(3.0), precision=lbm.FP32)
    sim.step(300)  # develop boundary layers so that every term of the collision is active
    f0, g0 = sim.get_populations()
    sim.step(1)
    f1, g1 = sim.get_populations()
    wf = oracle.weights_flow()
    wg = thermal_floor(q, p.cs2_phi, p.T_hot - p.T_cold)
    worst = 0.0
    for (i, j, k) in sample_nodes(N, 7 + q):
        fr, gr = p.cell_update(f0, g0, i, j, k)
        ef = np.abs(f1[:, k, j, i] - fr) / (FP32_REL * np.maximum(np.abs(fr), wf))
        eg = np.abs(g1[:, k, j, i] - gr) / (FP32_REL * np.maximum(np.abs(gr), wg))
        worst = max(worst, ef.max(), eg.max())
        assert ef.max() <= 1.0 and eg.max() <= 1.0, (i, j, k, ef.max(), eg.max())
    # properties that hold at any size: mass is conserved by the closed cavity
    assert abs(f1.sum() - f0.sum()) <= 1e-6 * f0.sum()
    assert np.isfinite(g1).all()
