"""The paper's Table 1 on the GPU: the 91^3 cubic cavity (the paper's grid) at
Ra = 1e3, 1e4, 1e5, Pr = 0.71, FP32, D3Q15 thermal lattice, run until the temperature
changes by less than 1e-6 over 100 steps, against the paper's LBM column and the
reference solution it quotes.

Tolerances, against the paper's LBM column; against the reference column the same
tolerance plus the paper's own deviation from it (the paper's LBM sits up to 4% from
the reference):
  Nu_mean  4% (at Ra = 1e5 this build is 3.3% above the paper and 0.8% below the
           reference);  u_max, w_max 3%;  Nu_max 5%;
  Nu_min   15%: it is the local Nu in the corner where the hot wall meets the adiabatic
           top wall, where the profile is steepest and the corner treatment matters most;
           the paper quotes it at z = 1, the last node of a half-way grid is 0.5/n below;
  positions 3 cells, as distance from the nearest wall (the maxima are broad and the
           paper's coordinates are quantised to 1/89)."""
import math

import pytest

from tests.golden_io import table1

pytestmark = pytest.mark.gpu

N = 91
STEADY = 1e-6        # max |dT| over 100 steps
MAX_STEPS = {1e3: 200_000, 1e4: 300_000, 1e5: 300_000}
TOL = {"Nu_mean": 0.04, "u_max": 0.03, "w_max": 0.03, "Nu_max": 0.05, "Nu_min": 0.15}
KEY = {"Nu_mean": "mid_mean", "u_max": "umax", "w_max": "wmax", "Nu_max": "mid_max",
       "Nu_min": "mid_min"}
POS = {"u_max": "umax_z", "w_max": "wmax_x", "Nu_max": "mid_max_z", "Nu_min": "mid_min_z"}


def run_to_steady(lbm, Ra, q=15):
    sim = lbm.LBM((N, N, N), q, Ra=Ra, Pr=0.71, Ma=0.05 * math.sqrt(3.0), precision=lbm.FP32,
                  residual_interval=100)
    while sim.steps_done < MAX_STEPS[Ra]:
        sim.step(2000)
        r = sim.residual()
        if 0 <= r < STEADY:
            break
    return sim, sim.residual()


@pytest.mark.timeout(900)
@pytest.mark.parametrize("Ra", [1e3, 1e4, 1e5])
def test_table1_at_91(Ra):
    import paper_1710_04751_gb300 as lbm
    sim, res = run_to_steady(lbm, Ra)
    nu = sim.nusselt()
    rows = {r["quantity"]: r for r in table1() if r["Ra"] == Ra}
    print(f"Ra={Ra:g} steps={sim.steps_done} residual={res:.2e} {nu}")
    assert 0 <= res < STEADY
    for q, tol in TOL.items():
        got, lbm_col, ref_col = nu[KEY[q]], rows[q]["lbm"], rows[q]["ref"]
        assert got == pytest.approx(lbm_col, rel=tol), (q, "paper LBM")
        own = abs(lbm_col - ref_col) / ref_col
        assert got == pytest.approx(ref_col, rel=tol + own), (q, "reference")
    near = lambda z: min(z, 1 - z)  # noqa: E731
    for q, key in POS.items():
        assert abs(near(nu[key]) - near(rows[q]["lbm_pos"])) <= 3.0 / N, q
    assert nu["hot_wall_mean"] == pytest.approx(nu["cold_wall_mean"], rel=1e-3)
