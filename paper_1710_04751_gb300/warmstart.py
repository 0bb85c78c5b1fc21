"""The learned warm start, end to end: solver-generated training data, training of the
network (include/lbm_net.h) on the GPU, and the comparison of warm-started and
cold-started runs to steady state.  Orchestration only: the solver steps, the network's
forward and backward passes and updates, the target extraction and the warm start all
run in liblbm.so; torch holds the device tensors and gathers training batches.

    data = generate(64, warmstart_samples(400, seed=1))
    netw = Net(n=64, max_batch=4)
    train(netw, data, epochs=30, batch=4)
    report = evaluate(netw, warmstart_samples(50, seed=2), n=64)
"""
import math
import time

import numpy as np

from . import net as _net
from .batch import Batch
from .lbm import FP32, LBM

U0_MA = 0.05 * math.sqrt(3.0)


def warmstart_samples(count, seed, Ra_range=(1e3, 1e6), Pr_range=(0.7, 7.0)):
    """(Ra, Pr) pairs, Ra and Pr log-uniform over their ranges (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    Ra = 10.0 ** rng.uniform(np.log10(Ra_range[0]), np.log10(Ra_range[1]), count)
    Pr = 10.0 ** rng.uniform(np.log10(Pr_range[0]), np.log10(Pr_range[1]), count)
    return [(float(a), float(p)) for a, p in zip(Ra, Pr)]


def _run_batch(n, samples, steady_tol, max_steps, warm=None, precision=FP32, chunk=10_000):
    """Advances one cubic cavity per sample to its own steady state (or max_steps / a
    divergence).  warm: None (cold start from rest) or (predictions [count][m^3][4], their
    grid m, rounds of consistent initialisation).  The wall time includes the warm start
    itself.  Returns the batch (still open), wall seconds and the status list."""
    import torch
    members = [{"grid": (n, n, n), "Ra": Ra, "Pr": Pr} for Ra, Pr in samples]
    b = Batch(members, precision=precision, residual_interval=100, steady_tol=steady_tol,
              Ma=U0_MA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if warm is not None:
        pred, m, rounds = warm
        for i in range(len(samples)):
            _net.warm_start(b.member(i), pred[i], m, rounds)
    while b.steps_done < max_steps and b.active_nodes > 0:
        b.step(min(chunk, max_steps - b.steps_done))
    torch.cuda.synchronize()
    return b, time.perf_counter() - t0, b.status()


def generate(n, samples, steady_tol=1e-6, max_steps=150_000):
    """Training data: every sample solved from rest to steady state at n^3 (FP32).
    Returns dict(scalars [k][2], targets CUDA [k][n^3][4], samples, steps) over the k
    samples that converged."""
    import torch
    b, secs, st = _run_batch(n, samples, steady_tol, max_steps)
    keep = [i for i, s in enumerate(st) if s["state"] == "converged"]
    targets = torch.empty((len(keep), n ** 3, 4), dtype=torch.float32, device="cuda")
    for j, i in enumerate(keep):
        targets[j] = _net.targets(b.member(i))
    b.close()
    return {"scalars": np.array([_net.encode(*samples[i]) for i in keep], dtype=np.float32),
            "targets": targets, "samples": [samples[i] for i in keep],
            "steps": [st[i]["steps"] for i in keep], "seconds": secs,
            "dropped": {"diverged": sum(s["state"] == "diverged" for s in st),
                        "not_converged": sum(s["state"] == "active" for s in st)}}


def train(netw, data, epochs, batch, seed=1, log_every=0, lr=1e-3, lr_final=1e-5):
    """Adam on shuffled mini-batches, the learning rate decaying geometrically from lr to
    lr_final over the epochs; returns the mean loss of every epoch."""
    import torch
    g = torch.Generator().manual_seed(seed)
    count = data["targets"].shape[0]
    history = []
    for ep in range(epochs):
        netw.set_lr(lr * (lr_final / lr) ** (ep / max(epochs - 1, 1)))
        perm = torch.randperm(count, generator=g).tolist()
        tot, nb = 0.0, 0
        for s in range(0, count - batch + 1, batch):
            idx = perm[s:s + batch]
            tot += netw.train_step(data["scalars"][idx], data["targets"][idx])
            nb += 1
        history.append(tot / max(nb, 1))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {history[-1]:.4e}", flush=True)
    return history


def predict(netw, samples):
    """Predictions [count][n^3][4] for (Ra, Pr) pairs, max_batch at a time."""
    import torch
    out = []
    for s in range(0, len(samples), netw.max_batch):
        chunk = samples[s:s + netw.max_batch]
        out.append(netw.forward([_net.encode(*p) for p in chunk]))
    return torch.cat(out, 0)


def evaluate(netw, samples, n, steady_tol=1e-6, max_steps=300_000, rounds=50):
    """Cold start and warm start (the network's prediction at its own grid, resampled to
    n^3, then `rounds` rounds of consistent initialisation) of every sample to its own
    steady state; steps (the warm ones including the rounds, an even number), wall time
    (the warm one including the prediction) and Nu of both."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pred = predict(netw, samples)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    rounds += rounds & 1
    res = {}
    pred_err = [None] * len(samples)
    for mode, warm in (("cold", None), ("warm", (pred, netw.n, rounds))):
        b, secs, st = _run_batch(n, samples, steady_tol, max_steps, warm=warm)
        nus = [b.member(i).nusselt()["hot_wall_mean"] if s["state"] == "converged" else None
               for i, s in enumerate(st)]
        if mode == "cold" and n == netw.n:  # prediction error against the steady fields
            for i, s in enumerate(st):
                if s["state"] == "converged":
                    t = _net.targets(b.member(i))
                    pred_err[i] = float((pred[i] - t).norm() / t.norm())
        res[mode] = {"seconds": secs, "status": st, "Nu": nus}
        b.close()
    rows = []
    for i, (Ra, Pr) in enumerate(samples):
        c, w = res["cold"]["status"][i], res["warm"]["status"][i]
        rows.append({"Ra": Ra, "Pr": Pr, "cold_state": c["state"], "warm_state": w["state"],
                     "cold_steps": c["steps"], "warm_steps": w["steps"] + rounds,
                     "Nu_cold": res["cold"]["Nu"][i], "Nu_warm": res["warm"]["Nu"][i],
                     "pred_rel_err": pred_err[i]})
    both = [r for r in rows if r["cold_state"] == "converged" and r["warm_state"] == "converged"]
    summary = {
        "n": n, "samples": len(samples), "both_converged": len(both), "init_rounds": rounds,
        "cold_seconds": round(res["cold"]["seconds"], 2),
        "warm_seconds": round(res["warm"]["seconds"] + t_pred, 2),
        "prediction_seconds": round(t_pred, 3),
    }
    if both:
        cs = np.array([r["cold_steps"] for r in both], dtype=float)
        ws = np.array([r["warm_steps"] for r in both], dtype=float)
        err = np.array([abs(r["Nu_warm"] - r["Nu_cold"]) / r["Nu_cold"] for r in both])
        summary.update({
            "steps_cold_median": float(np.median(cs)), "steps_warm_median": float(np.median(ws)),
            "steps_saved_mean_frac": float(np.mean(1 - ws / cs)),
            "Nu_warm_vs_cold_max_rel": float(err.max()),
            "Nu_warm_vs_cold_mean_rel": float(err.mean()),
        })
        pe = [r["pred_rel_err"] for r in both if r["pred_rel_err"] is not None]
        if pe:
            summary["pred_rel_err_median"] = float(np.median(pe))
    return {"summary": summary, "rows": rows}


def fp64_reference(samples, n, steady_tol=1e-7, max_steps=300_000):
    """Steady hot-wall Nu of each sample from the FP64 solver (step-for-step equal to the
    FP64 oracle to 1e-12), one context at a time; None where it does not converge."""
    out = []
    for Ra, Pr in samples:
        sim = LBM((n, n, n), 15, Ra=Ra, Pr=Pr, Ma=U0_MA, precision=0, residual_interval=100)
        res = -1.0
        while sim.steps_done < max_steps:
            sim.step(5000)
            res = sim.residual()
            if 0 <= res < steady_tol:
                break
        out.append(sim.nusselt()["hot_wall_mean"] if 0 <= res < steady_tol else None)
        sim.close()
    return out


def nu_error_vs_fp64(report, n, count, steady_tol=1e-6):
    """The final hot-wall Nu of the warm-started (and the cold-started) FP32 runs of the
    first `count` held-out cases where both converged, against the FP64 solver run to the
    same convergence test from rest (the FP64 solver follows the FP64 oracle step for step
    to 1e-12)."""
    rows = [r for r in report["rows"] if r["cold_state"] == "converged" and r["warm_state"] == "converged"]
    rows = rows[:count]
    ref = fp64_reference([(r["Ra"], r["Pr"]) for r in rows], n, steady_tol=steady_tol)
    out = []
    for r, nu64 in zip(rows, ref):
        if nu64 is None:
            continue
        out.append({"Ra": r["Ra"], "Pr": r["Pr"], "Nu_fp64": nu64,
                    "warm_rel": (r["Nu_warm"] - nu64) / nu64, "cold_rel": (r["Nu_cold"] - nu64) / nu64})
    summary = {"cases": len(out)}
    if out:
        w = np.array([abs(o["warm_rel"]) for o in out])
        c = np.array([abs(o["cold_rel"]) for o in out])
        summary.update({"warm_max_rel": float(w.max()), "warm_mean_rel": float(w.mean()),
                        "cold_max_rel": float(c.max()), "cold_mean_rel": float(c.mean())})
    return {"summary": summary, "rows": out}


def experiment(n_train=64, count_train=400, count_test=50, n_big=128, count_big=8, epochs=40,
               batch=4, rounds=50, seed=1, steady_tol=1e-6, count_fp64=12, log=print):
    """The learned warm start end to end: `count_train` steady states at n_train^3 with Ra
    log-uniform in [1e3, 1e6] and Pr log-uniform in [0.7, 7] (seed), the network trained on
    them, and cold against warm starts on `count_test` held-out samples at n_train^3 and
    `count_big` of them at n_big^3 (the prediction resampled trilinearly); the final Nu of
    `count_fp64` of the n_train^3 cases against the FP64 solver."""
    import torch
    from .net import Net
    t0 = time.perf_counter()
    data = generate(n_train, warmstart_samples(count_train, seed), steady_tol=steady_tol)
    t_gen = time.perf_counter() - t0
    log(f"generated {len(data['samples'])} / {count_train} steady states in {t_gen:.1f} s "
        f"(dropped {data['dropped']})")
    netw = Net(n=n_train, max_batch=batch, seed=seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = train(netw, data, epochs, batch, seed=seed, log_every=max(1, epochs // 8))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    test = warmstart_samples(count_test, seed + 1000)
    rep = evaluate(netw, test, n_train, steady_tol=steady_tol, rounds=rounds)
    log(f"{n_train}^3: {rep['summary']}")
    big = None
    if count_big:
        big = evaluate(netw, test[:count_big], n_big, steady_tol=steady_tol, rounds=rounds)
        log(f"{n_big}^3: {big['summary']}")
    fp64 = None
    if count_fp64:
        fp64 = nu_error_vs_fp64(rep, n_train, count_fp64, steady_tol=steady_tol)
        log(f"Nu against the FP64 solver ({n_train}^3): {fp64['summary']}")
    out = {"train": {"samples": len(data["samples"]), "dropped": data["dropped"],
                     "generate_seconds": round(t_gen, 1), "epochs": epochs, "batch": batch,
                     "train_seconds": round(t_train, 1), "loss_first": hist[0],
                     "loss_last": hist[-1], "params": netw.param_count},
           "test": rep, "big": big, "fp64": fp64}
    return out, netw


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start: generate, train, evaluate")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--test", type=int, default=50)
    ap.add_argument("--big", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--rounds", type=int, default=50)
    ap.add_argument("--fp64", type=int, default=12, help="held-out cases checked against the FP64 solver")
    ap.add_argument("--save", default=None, help="write the trained parameters (float32) here")
    a = ap.parse_args()
    res, netw = experiment(a.n, a.train, a.test, 2 * a.n, a.big, a.epochs, rounds=a.rounds,
                           count_fp64=a.fp64)
    if a.save:
        netw.get_params().tofile(a.save)
    print(json.dumps(res))
