"""The paper's Table 1 (Sec. 3) on the GPU at several resolutions: the differentially heated
cubic cavity at Ra = 1e3, 1e4, 1e5, Pr = 0.71, U0 = 0.05, D3Q15 flow + D3Q15 scalar, from
rest until max |dT| over 100 steps falls below 1e-6 (the first steady plateau), then the
symmetry-plane quantities of Table 1: u_max, w_max, Nu_max, Nu_min, Nu_mean and their
positions.  A grid-convergence study of those quantities tells a discretisation error
(which shrinks with the grid) from a reading of the paper (which does not).

    python -m paper_1710_04751_gb300.table1 [--grids 91 128 182] [--Ra 1e3 1e4 1e5]
        [--e4-modes 0 1] [--fp64-grid 91] [--json out.json]

Every run is FP32 with the fourth-order flow equilibrium of reading R1 (e4_mode 0),
unless listed in --e4-modes (runs of the first grid with the other reading) or
--fp64-grid (the same runs in FP64 on that grid).  Prints one JSON object per run and a
Markdown table against the paper's LBM column.
"""
import argparse
import json
import math
import time

from . import lbm as _lbm

PR, U0 = 0.71, 0.05
STEADY = 1e-6
# Table 1 of the paper: its LBM column on 91^3 (quantity -> Ra -> value)
PAPER = {
    "u_max": {1e3: 0.1308, 1e4: 0.1965, 1e5: 0.1441},
    "w_max": {1e3: 0.1308, 1e4: 0.2232, 1e5: 0.2447},
    "Nu_max": {1e3: 1.4170, 1e4: 3.5815, 1e5: 7.745},
    "Nu_min": {1e3: 0.730, 1e4: 0.5925, 1e5: 0.772},
    "Nu_mean": {1e3: 1.0977, 1e4: 2.2647, 1e5: 4.4595},
}
KEY = {"u_max": "umax", "w_max": "wmax", "Nu_max": "mid_max", "Nu_min": "mid_min",
       "Nu_mean": "mid_mean"}
POS = {"u_max": "umax_z", "w_max": "wmax_x", "Nu_max": "mid_max_z", "Nu_min": "mid_min_z"}


def run(n, Ra, precision="FP32", e4_mode=0, max_steps=None, chunk=2000, lattice=15,
        adiabatic_mode=_lbm.ADIABATIC_SPECULAR):
    """One cavity from rest to its first steady plateau; returns the Table 1 quantities."""
    max_steps = max_steps or int(6000 * n)
    sim = _lbm.LBM((n, n, n), lattice, Ra=Ra, Pr=PR, Ma=U0 * math.sqrt(3.0),
                   precision=getattr(_lbm, precision), e4_mode=e4_mode,
                   adiabatic_mode=adiabatic_mode, residual_interval=100)
    t0 = time.perf_counter()
    res = -1.0
    while sim.steps_done < max_steps:
        sim.step(chunk)
        res = sim.residual()
        if 0 <= res < STEADY:
            break
    dt = time.perf_counter() - t0
    nu = sim.nusselt()
    out = {"n": n, "Ra": Ra, "precision": precision, "e4_mode": e4_mode, "lattice": lattice,
           "adiabatic_mode": adiabatic_mode,
           "steps": sim.steps_done, "seconds": round(dt, 2), "residual_per_100": res,
           "steady": bool(0 <= res < STEADY)}
    for q, k in KEY.items():
        out[q] = nu[k]
    for q, k in POS.items():
        out[q + "_pos"] = nu[k]
    out["Nu_hot_wall"] = nu["hot_wall_mean"]
    sim.close()
    return out


def markdown(rows):
    lines = ["| n | Ra | form | steps | " + " | ".join(PAPER) + " |",
             "|---|---|---|---|" + "---|" * len(PAPER)]
    for r in rows:
        cells = []
        for q in PAPER:
            ref = PAPER[q][r["Ra"]]
            cells.append(f"{r[q]:.4f} ({100 * (r[q] - ref) / ref:+.1f}%)")
        form = r["precision"] + ("" if r["e4_mode"] == 0 else " E=rho/9")
        form += "" if r.get("lattice", 15) == 15 else " D3Q7"
        form += "" if r.get("adiabatic_mode", 1) == 1 else " bounce-back"
        lines.append(f"| {r['n']} | {r['Ra']:g} | {form} | {r['steps']} | " + " | ".join(cells) + " |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--grids", type=int, nargs="+", default=[91, 128, 182])
    ap.add_argument("--Ra", type=float, nargs="+", default=[1e3, 1e4, 1e5])
    ap.add_argument("--e4-modes", type=int, nargs="*", default=[1])
    ap.add_argument("--fp64-grid", type=int, default=91)
    ap.add_argument("--fp64-Ra", type=float, nargs="*", default=[1e4, 1e5])
    ap.add_argument("--variants", action="store_true",
                    help="also the D3Q7 scalar lattice and the bounce-back adiabatic rule on every grid")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    rows = []
    plan = [(n, Ra, "FP32", 0) for n in args.grids for Ra in args.Ra]
    plan += [(args.grids[0], Ra, "FP32", m) for m in args.e4_modes if m != 0 for Ra in args.Ra]
    if args.fp64_grid:
        plan += [(args.fp64_grid, Ra, "FP64", 0) for Ra in args.fp64_Ra]
    plan = [(n, Ra, prec, mode, 15, 1) for n, Ra, prec, mode in plan]
    if args.variants:
        plan += [(n, Ra, "FP32", 0, 7, 1) for n in args.grids for Ra in args.Ra]
        plan += [(n, Ra, "FP32", 0, 15, 0) for n in args.grids for Ra in args.Ra]
    for n, Ra, prec, mode, q, am in plan:
        r = run(n, Ra, prec, mode, lattice=q, adiabatic_mode=am)
        rows.append(r)
        print(json.dumps(r), flush=True)
    print(markdown(rows), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()
