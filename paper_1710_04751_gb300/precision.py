"""The 16-bit storage forms against FP32 and FP64 runs of the same cavity.

The precision form stores populations as FP16 or BF16 deviations from the local rest state
(w_a for the flow, w^phi_a T_node for the scalar) and computes in FP32; the Nusselt and
residual reductions are FP64 in every form.  This study reports what that costs in
accuracy and what it saves in time:

    python -m paper_1710_04751_gb300.precision [--n 256] [--Ra 1e6] [--ref-n 64]
        [--ref-Ra 1e5] [--max-steps 400000] [--fp64-seconds 60]

Part 1, the large cavity (default 256^3, Ra = 1e6, Pr = 0.71, U0 = 0.05, D3Q15 flow and
scalar): FP32 from rest to the steady state, FP16 and BF16 from rest for the same number of
steps (steps, wall seconds, Nusselt numbers, peak velocities, mid-plane fields; 16-bit
against FP32),
and an FP64 run of as many steps as fit in --fp64-seconds, against which the three are
compared after the same number of steps.

Part 2, the reference cavity (default 64^3, Ra = 1e5): FP64 to the steady state, FP32,
FP16 and BF16 for the same number of steps; every form against FP64.

Steady state of the reference form: the hot-wall Nusselt number changes by less than 1e-5
(relative) over 10 000 steps (run_to_steady).  The 16-bit forms cannot end on a test of
their own: their max |dT| per 100 steps has a rounding floor (about 2e-5 in FP16, 2e-4 in
BF16) and their face-averaged Nusselt number carries rounding noise of about 1e-5, so they
run the reference form's number of steps.

Mid-plane fields: T and u on the symmetry plane y = L/2 (the mean of the two straddling
layers for even n), errors as max and RMS of |difference| over the plane, T in units of
the wall temperature difference and u in units of the buoyancy velocity U0.  Prints one
JSON object.
"""
import argparse
import json
import math
import time

import numpy as np

from . import lbm as _lbm

PR, U0 = 0.71, 0.05
NU_KEYS = ("hot_wall_mean", "cold_wall_mean", "mid_mean", "mid_max", "mid_min", "umax", "wmax")
FORMS = ("FP64", "FP32", "FP16_DEV", "BF16_DEV")


def _new(n, Ra, form, q=15):
    return _lbm.LBM((n, n, n), q, Ra=Ra, Pr=PR, Ma=U0 * math.sqrt(3.0),
                    precision=getattr(_lbm, form), residual_interval=100)


def mid_plane(sim):
    """T and u / U0 on the symmetry plane y = L/2, arrays indexed [z, x]."""
    fl = sim.fields()
    ny = fl["T"].shape[1]
    js = [ny // 2 - 1, ny // 2] if ny % 2 == 0 else [ny // 2]
    out = {k: fl[k][:, js, :].mean(axis=1) for k in ("T", "ux", "uy", "uz")}
    for k in ("ux", "uy", "uz"):
        out[k] = out[k] / U0
    return out


def plane_errors(a, b):
    """Max and RMS differences of the mid-plane fields a - b (T in units of dT, u in U0)."""
    out = {}
    dT = a["T"] - b["T"]
    du = np.sqrt(sum((a[k] - b[k]) ** 2 for k in ("ux", "uy", "uz")))
    out["T_max"] = float(np.abs(dT).max())
    out["T_rms"] = float(np.sqrt((dT ** 2).mean()))
    out["u_max"] = float(du.max())
    out["u_rms"] = float(np.sqrt((du ** 2).mean()))
    return out


def nu_errors(a, b):
    """Relative differences of the Nusselt numbers and peak velocities a against b."""
    return {k: float((a[k] - b[k]) / b[k]) if b[k] != 0 else float(a[k] - b[k]) for k in NU_KEYS}


def run_to_steady(n, Ra, form, max_steps, nu_tol=1e-5, window=10_000, chunk=2000):
    """From rest until the hot-wall Nusselt number changes by less than nu_tol (relative)
    over `window` steps, or max_steps.  The same test ends every storage form: the
    residual max |dT| per 100 steps has a rounding floor of about 2e-5 in FP16 and 2e-4 in
    BF16, so a residual threshold below those is never met; it is reported too."""
    import torch
    sim = _new(n, Ra, form)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, history = -1.0, []
    diverged = converged = False
    while sim.steps_done < max_steps:
        try:
            sim.step(chunk)
        except _lbm.LBMError as e:
            if e.code != _lbm.LBM_EDIVERGED:
                raise
            diverged = True
            break
        res = sim.residual()
        history.append((sim.steps_done, sim.nusselt()["hot_wall_mean"]))
        back = [h for s_, h in history if s_ <= sim.steps_done - window]
        if back and abs(history[-1][1] - back[-1]) <= nu_tol * abs(history[-1][1]):
            converged = True
            break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nu = sim.nusselt()
    rec = {"form": form, "converged": converged, "diverged": diverged, "steps": sim.steps_done,
           "seconds": round(dt, 3), "residual_per_100": res,
           "criterion": f"|dNu_hot|/Nu_hot < {nu_tol:g} over {window} steps",
           "nu": {k: nu[k] for k in NU_KEYS},
           "positions": {k: nu[k] for k in ("mid_max_z", "mid_min_z", "umax_z", "wmax_x")}}
    return sim, rec


def run_steps(n, Ra, form, steps, chunk=2000):
    """From rest for exactly `steps` steps, in the chunks run_to_steady takes."""
    import torch
    sim = _new(n, Ra, form)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while sim.steps_done < steps:
        sim.step(min(chunk, steps - sim.steps_done))
        sim.residual()
        sim.nusselt()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    nu = sim.nusselt()
    rec = {"form": form, "steps": sim.steps_done, "seconds": round(dt, 3),
           "residual_per_100": sim.residual(), "criterion": "the reference form's step count",
           "nu": {k: nu[k] for k in NU_KEYS},
           "positions": {k: nu[k] for k in ("mid_max_z", "mid_min_z", "umax_z", "wmax_x")}}
    return sim, rec


def fixed_steps(n, Ra, form, steps):
    import torch
    sim = _new(n, Ra, form)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(steps)
    torch.cuda.synchronize()
    return sim, time.perf_counter() - t0


def large_cavity(n, Ra, max_steps, fp64_seconds):
    out = {"grid": n, "Ra": Ra, "Pr": PR, "U0": U0, "lattice": "D3Q15+D3Q15"}
    steady, planes = {}, {}
    # FP32 runs to its steady state; the 16-bit forms run the same number of steps (their
    # rounding noise makes a convergence test of their own unreliable)
    sim, rec = run_to_steady(n, Ra, "FP32", max_steps)
    steady["FP32"], planes["FP32"] = rec, mid_plane(sim)
    sim.close()
    S = rec["steps"]
    for form in ("FP16_DEV", "BF16_DEV"):
        sim, rec = run_steps(n, Ra, form, S)
        steady[form], planes[form] = rec, mid_plane(sim)
        sim.close()
    for rec in steady.values():
        rec["mlups"] = round(n ** 3 * rec["steps"] / rec["seconds"] / 1e6, 1)
    out["steady"] = steady
    ref = steady["FP32"]
    out["steady_vs_fp32"] = {
        f: {"nu": nu_errors(steady[f]["nu"], ref["nu"]), "plane": plane_errors(planes[f], planes["FP32"]),
            "time_ratio": round(steady[f]["seconds"] / ref["seconds"], 4)}
        for f in ("FP16_DEV", "BF16_DEV")}
    # FP64 for as many steps as fit in the time budget, then every form after those steps
    probe, t = fixed_steps(n, Ra, "FP64", 20)
    probe.close()
    k = max(100, int(fp64_seconds / max(t / 20, 1e-6)) // 100 * 100)
    sims = {}
    for form in FORMS:
        sim, t = fixed_steps(n, Ra, form, k)
        sims[form] = (sim.nusselt(), mid_plane(sim), t)
        sim.close()
    ref_nu, ref_plane, _ = sims["FP64"]
    out["fixed_steps_vs_fp64"] = {
        "steps": k, "fp64_ms_per_step": round(sims["FP64"][2] / k * 1e3, 3),
        **{f: {"nu": nu_errors(sims[f][0], ref_nu), "plane": plane_errors(sims[f][1], ref_plane),
               "ms_per_step": round(sims[f][2] / k * 1e3, 4)} for f in FORMS[1:]}}
    return out


def reference_cavity(n, Ra, ref_max_steps):
    out = {"grid": n, "Ra": Ra, "Pr": PR, "U0": U0, "lattice": "D3Q15+D3Q15"}
    steady, planes = {}, {}
    sim, rec = run_to_steady(n, Ra, "FP64", ref_max_steps)
    steady["FP64"], planes["FP64"] = rec, mid_plane(sim)
    sim.close()
    for form in FORMS[1:]:
        sim, rec = run_steps(n, Ra, form, steady["FP64"]["steps"])
        steady[form], planes[form] = rec, mid_plane(sim)
        sim.close()
    out["steady"] = steady
    out["vs_fp64"] = {f: {"nu": nu_errors(steady[f]["nu"], steady["FP64"]["nu"]),
                          "plane": plane_errors(planes[f], planes["FP64"])} for f in FORMS[1:]}
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--Ra", type=float, default=1e6)
    ap.add_argument("--ref-n", type=int, default=64)
    ap.add_argument("--ref-Ra", type=float, default=1e5)
    ap.add_argument("--max-steps", type=int, default=400_000)
    ap.add_argument("--ref-max-steps", type=int, default=120_000,
                    help="cap of the reference runs (the 64^3 Ra = 1e5 cavity leaves its steady "
                         "state after about 1.3e5 steps)")
    ap.add_argument("--fp64-seconds", type=float, default=60.0)
    ap.add_argument("--skip-large", action="store_true")
    ap.add_argument("--skip-ref", action="store_true")
    args = ap.parse_args(argv)
    _lbm.load()
    res = {}
    if not args.skip_ref:
        res["reference"] = reference_cavity(args.ref_n, args.ref_Ra, args.ref_max_steps)
        print(json.dumps({"reference": res["reference"]}), flush=True)
    if not args.skip_large:
        res["large"] = large_cavity(args.n, args.Ra, args.max_steps, args.fp64_seconds)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
