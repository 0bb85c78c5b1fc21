"""Benchmark of the fused cascaded thermal LBM step on GB300.

Workload: the differentially heated cubic cavity at 128^3, Ra = 1e5, Pr = 0.71,
U0 = 0.05, FP32 populations, D3Q15 flow + D3Q15 thermal (headline) and D3Q15 flow +
D3Q7 thermal (variant).  A bench "step" is one time step: one fused stream-and-collide
kernel over the whole grid, plus the residual / NaN reduction every 100 steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU) every rank
advances its own cavity (the method has no exchange between independent cavities) and
the value is the whole-job throughput over the slowest rank.
"""
import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS & % HBM roofline; time-to-steady Nu at Ra=1e5 vs plain FP32"
N_GRID, RA, PR, U0 = 128, 1e5, 0.71, 0.05
RESIDUAL_INTERVAL = 100
KERNEL_STEPS = 1000  # steps per kernel-timing graph
# algorithmic bytes per node update: every population read once and written once; the
# 16-bit forms also read and write the FP32 node temperature their thermal deviations use
def bytes_per_node(q, storage_bytes=4):
    return 2 * (15 + q) * storage_bytes + (2 * 4 if storage_bytes == 2 else 0)


BYTES_PER_NODE = {15: bytes_per_node(15), 7: bytes_per_node(7)}


# ----------------------------------------------------------------------------------
# distributed helpers (one process per GPU; tested with gloo on CPU)
# ----------------------------------------------------------------------------------

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def init_dist(world, backend):
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist if world > 1 else None


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, value, device=None):
    """Max of a float over all ranks (the slowest rank sets the job time)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------

CLOCK_LOAD_STEPS = 6000  # about 0.5 s of 128^3 steps

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return self
        self.proc = subprocess.Popen(
            [exe, "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
             "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[4:8]):
                if flag.lower() == "active":
                    reasons.add(name)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------

def time_steps(sim, steps, stream):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    sim.step(steps)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def run_variant(lbm, q, steps, warmup, dist, device, clocks=None, precision=None, n=N_GRID):
    import torch
    n3 = n ** 3
    precision = lbm.FP32 if precision is None else precision
    stream = torch.cuda.current_stream(device)
    sim = lbm.LBM((n,) * 3, q, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0), precision=precision,
                  residual_interval=RESIDUAL_INTERVAL)
    sim.step(warmup)
    torch.cuda.synchronize()
    barrier(dist)
    if clocks is not None:
        # the timed region is a few ms, shorter than nvidia-smi's sampling period: the
        # sampler runs over a window of back-to-back steps (about 0.5 s each side) that
        # encloses it, so that its samples are taken under the same load
        clocks.start()
        time.sleep(0.15)
        sim.step(CLOCK_LOAD_STEPS)
        torch.cuda.synchronize()
    elapsed = time_steps(sim, steps, stream)
    if clocks is not None:
        sim.step(CLOCK_LOAD_STEPS)
        torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    if clk is not None:
        clk["window"] = f"{CLOCK_LOAD_STEPS} steps before and after the timed region"
    barrier(dist)
    elapsed_max = max_over_ranks(dist, elapsed, device)
    nu = sim.nusselt()
    residual = sim.residual()

    # the step kernel for the roofline, as lbm_step runs it: one CUDA graph of KSTEPS steps
    # (its single residual check adds < 0.05%); the first call captures the graph
    ksteps = KERNEL_STEPS
    kern = lbm.LBM((n,) * 3, q, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0), precision=precision,
                   residual_interval=ksteps)
    kern.step(ksteps)
    t_kernel = time_steps(kern, ksteps, stream) / ksteps
    kern.close()
    return dict(sim=sim, elapsed=elapsed_max, mlups=n3 * steps / elapsed_max / 1e6,
                t_kernel=t_kernel, nu=nu, residual=residual, clocks=clk,
                launches=steps + steps // RESIDUAL_INTERVAL)


def e2e_variant(lbm, q, reps, device):
    """Through the C ABI with host buffers: upload the state from pinned host memory,
    advance one residual interval, read Nu and the residual back.  Per repetition.  The
    upload goes through the native-precision call (FP32 values, no conversion pass); the
    same measurement with the FP64 call is reported beside it."""
    import torch
    n = N_GRID
    sim = lbm.LBM((n,) * 3, q, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0), precision=lbm.FP32,
                  residual_interval=RESIDUAL_INTERVAL)
    out = {}
    for kind, dtype in (("native", torch.float32), ("fp64", torch.float64)):
        f_host = torch.empty((15, n, n, n), dtype=dtype, pin_memory=True).numpy()
        g_host = torch.empty((q, n, n, n), dtype=dtype, pin_memory=True).numpy()
        if kind == "native":
            sim.get_populations_native(f_host, g_host)
            upload = lambda: sim.set_populations_native(f_host, g_host)  # noqa: E731
        else:
            f, g = sim.get_populations()
            f_host[...] = f
            g_host[...] = g
            upload = lambda: sim.set_populations(f_host, g_host)  # noqa: E731
        upload()
        sim.step(RESIDUAL_INTERVAL)
        sim.nusselt()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            upload()
            sim.step(RESIDUAL_INTERVAL)
            sim.nusselt()
            sim.residual()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        lups = n ** 3 * RESIDUAL_INTERVAL * reps
        out[kind] = dict(value=lups / dt / 1e6, unit="MLUPS",
                         h2d_bytes_per_step=(15 + q) * n ** 3 * f_host.itemsize / RESIDUAL_INTERVAL,
                         d2h_bytes_per_step=(11 * 8) / RESIDUAL_INTERVAL)
    sim.close()
    res = dict(out["native"])
    res.update(lbm_steps_per_transfer=RESIDUAL_INTERVAL,
               note="per step: H2D of the FP32 state from pinned memory (lbm_set_populations_native), "
                    "100 fused steps, D2H of Nu; bytes amortised per time step",
               fp64_upload={k: out["fp64"][k] for k in ("value", "unit", "h2d_bytes_per_step")})
    return res


def time_to_steady(lbm, q, max_steps, threshold=1e-6, chunk=1000):
    """Plain FP32 method from the initial state until max |dT| over 100 steps falls
    below `threshold` (128^3, Ra = 1e5): steps, wall seconds and the steady Nu.  In FP32
    the rounding noise of max |dT| over 100 steps on 2M nodes is about 3e-7, so the
    threshold is 1e-6 (1e-7 is only reachable in FP64)."""
    import torch
    sim = lbm.LBM((N_GRID,) * 3, q, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0), precision=lbm.FP32,
                  residual_interval=RESIDUAL_INTERVAL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = -1.0
    while sim.steps_done < max_steps:
        sim.step(chunk)
        res = sim.residual()
        if 0 <= res < threshold:
            break
    dt = time.perf_counter() - t0
    nu = sim.nusselt()
    steps = sim.steps_done
    sim.close()
    return {"converged": bool(0 <= res < threshold), "steps": steps,
            "seconds": round(dt, 2), "residual_per_100": res, "threshold": threshold,
            "Nu_mean_mid": nu["mid_mean"], "Nu_hot": nu["hot_wall_mean"],
            "Nu_max": nu["mid_max"], "Nu_min": nu["mid_min"], "u_max": nu["umax"],
            "w_max": nu["wmax"]}


def time_to_steady_16bit(lbm, q, fp32, chunk=1000):
    """The 16-bit storage forms on the same cavity and initial state, for the number of steps
    the plain FP32 run needed (their max |dT| per 100 steps has a rounding floor above the
    threshold, about 2e-5 in FP16 and 2e-4 in BF16, so they cannot end on it): wall seconds
    against FP32's and their Nusselt numbers and peak velocities against FP32's."""
    import torch
    out = {}
    keys = (("Nu_mean_mid", "mid_mean"), ("Nu_hot", "hot_wall_mean"), ("Nu_max", "mid_max"),
            ("Nu_min", "mid_min"), ("u_max", "umax"), ("w_max", "wmax"))
    for name in ("FP16_DEV", "BF16_DEV"):
        sim = lbm.LBM((N_GRID,) * 3, q, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0),
                      precision=getattr(lbm, name), residual_interval=RESIDUAL_INTERVAL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while sim.steps_done < fp32["steps"]:
            sim.step(min(chunk, fp32["steps"] - sim.steps_done))
            sim.residual()
        dt = time.perf_counter() - t0
        nu = sim.nusselt()
        sim.close()
        out[name] = {"steps": fp32["steps"], "seconds": round(dt, 2),
                     "time_vs_fp32": round(dt / fp32["seconds"], 4),
                     **{k: nu[src] for k, src in keys},
                     "rel_diff_vs_fp32": {k: round((nu[src] - fp32[k]) / fp32[k], 5) for k, src in keys}}
    return out


def batch_variant(lbm, steps, warmup, peak, converge_steps=0):
    """The batched form: 64 cavities (edge 32/48/64/96, Ra log-uniform in [1e3, 1e6],
    Pr in {0.71, 1, 7}, seed 1), FP32, D3Q15 + D3Q15, one persistent kernel launch per
    step captured in graphs of 100 steps, tiling chosen by the autotuner; against the
    same members advanced with one single-cavity kernel launch per member and step.
    Throughput counts the node updates actually done (members that diverge stop)."""
    import torch
    from paper_1710_04751_gb300.workloads import cavity_sweep
    members = cavity_sweep(64, seed=1)
    b = lbm.Batch(members, precision=lbm.FP32, residual_interval=RESIDUAL_INTERVAL,
                  autotune_steps=0)
    trials = b.autotune(trial_steps=5)
    tuned_nodes = b.active_nodes  # every member is active while the tuner times the kernels
    stream = torch.cuda.current_stream()
    ncell = [m["grid"][0] ** 3 for m in members]

    def timed(mode, n):
        before = [s["steps"] for s in b.status()]
        t = time_steps_mode(b, n, stream, mode)
        after = [s["steps"] for s in b.status()]
        lups = sum(c * (a - s0) for c, a, s0 in zip(ncell, after, before))
        return lups / t / 1e6, t

    b.step(warmup)
    res = {}
    for mode in ("graph", "launch", "sequential"):
        mlups, t = timed(mode, steps)
        res[mode] = {"value": round(mlups, 1), "unit": "MLUPS", "seconds": round(t, 4)}
    st = b.status()
    tiling = b.tiling
    best = min(trials, key=lambda t: t["ms_per_step"])
    bpn = bytes_per_node(15)
    achieved = bpn * tuned_nodes / (best["ms_per_step"] * 1e-3) / 1e9
    out = {
        "workload": "64 cubic cavities, edge from {32,48,64,96}, Ra log-uniform [1e3,1e6], "
                    "Pr from {0.71,1,7}, seed 1; FP32, D3Q15+D3Q15",
        "nodes": sum(ncell), "steps": steps, "warmup": warmup,
        "batched_graph": res["graph"], "batched_launch_per_step": res["launch"],
        "sequential_per_cavity_launches": res["sequential"],
        "speedup_vs_sequential": round(res["graph"]["value"] / res["sequential"]["value"], 3),
        "tiling": tiling,
        "autotune": [{k: t[k] for k in ("threads", "min_blocks", "mapping", "blocks_per_sm", "tile_factor")}
                     | {"ms": round(t["ms_per_step"], 4)} for t in trials],
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "kernel": "batch_step_kernel<float,15>",
                     "bytes_per_node": bpn, "kernel_ms": round(best["ms_per_step"], 4),
                     "nodes_per_launch": tuned_nodes},
        "states_after": {k: sum(1 for s in st if s["state"] == k)
                         for k in ("active", "converged", "diverged")},
    }
    b.close()
    if converge_steps > 0:
        out["to_convergence"] = batch_to_convergence(lbm, members, converge_steps)
        out["to_convergence_sequential"] = batch_to_convergence(lbm, members, converge_steps,
                                                                mode="sequential")
    return out


def slab_variant(lbm, steps, warmup, device, undivided_ms):
    """The same 128^3 cavity decomposed into z-slabs with a halo exchange after every step
    (one GPU: the decomposition's own cost, the extra halo planes and the exchange kernel)."""
    import torch
    from paper_1710_04751_gb300 import slabs
    stream = torch.cuda.current_stream(device)
    out = {}
    for nslabs in (2, 4):
        dec = slabs.Slabs((N_GRID,) * 3, nslabs, 15, Ra=RA, Pr=PR, Ma=U0 * math.sqrt(3.0),
                          residual_interval=RESIDUAL_INTERVAL)
        dec.step(warmup)
        t = time_steps(dec, steps, stream)
        ms = t / steps * 1e3
        out[f"{nslabs} slabs"] = {
            "value": round(N_GRID ** 3 * steps / t / 1e6, 1), "unit": "MLUPS", "steps": steps,
            "ms_per_step": round(ms, 5), "undivided_ms_per_step": round(undivided_ms, 5),
            "time_vs_undivided": round(ms / undivided_ms, 4),
            "halo_bytes_per_step": dec.halo_bytes, "kernel_launches_per_step": nslabs + 1}
        dec.close()
    return out


def time_steps_mode(b, steps, stream, mode):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    b.step(steps, mode=mode)
    end.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(end) / 1e3


def batch_to_convergence(lbm, members, max_steps, tol=1e-6, mode="graph"):
    """Every member of the sweep from rest until its own max |dT| over 100 steps falls
    below tol (FP32 floor: see time_to_steady) or it diverges, up to max_steps; `mode`
    "sequential" advances the same members with one single-cavity launch per member and
    step (the plain method, cavity after cavity) under the same stopping rule."""
    import torch
    b = lbm.Batch(members, precision=lbm.FP32, residual_interval=RESIDUAL_INTERVAL,
                  steady_tol=tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_at = []
    while b.steps_done < max_steps and b.active_nodes > 0:
        b.step(min(10_000, max_steps - b.steps_done), mode=mode)
        done_at.append((b.steps_done, round(time.perf_counter() - t0, 2), b.active_nodes))
    dt = time.perf_counter() - t0
    st = b.status()
    conv = [s["steps"] for s in st if s["state"] == "converged"]
    nus = []
    for i, s in enumerate(st):
        if s["state"] == "converged":
            nu = b.member(i).nusselt()
            nus.append({"n": members[i]["grid"][0], "Ra": round(members[i]["Ra"], 1),
                        "Pr": members[i]["Pr"], "steps": s["steps"],
                        "Nu_hot": round(nu["hot_wall_mean"], 5)})
    ncell = [m["grid"][0] ** 3 for m in members]
    lups = sum(c * s["steps"] for c, s in zip(ncell, st))
    b.close()
    return {"mode": mode, "tol": tol, "max_steps": max_steps, "seconds": round(dt, 2),
            "converged": len(conv), "diverged": sum(1 for s in st if s["state"] == "diverged"),
            "active": sum(1 for s in st if s["state"] == "active"),
            "steps_min_median_max": [min(conv), sorted(conv)[len(conv) // 2], max(conv)] if conv else None,
            "node_updates": lups, "mlups": round(lups / dt / 1e6, 1),
            "progress": done_at[:: max(1, len(done_at) // 12)], "converged_members": nus}


def measured_peak_tflops():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def net_variant():
    """The warm-start network's tensor-core path: tcgen05 GEMM throughput (a large GEMM and
    the network's own convolution shapes at 64^3, batch 2) against the measured BF16
    peak, and the time of one training step and one forward pass at 64^3."""
    import torch
    from paper_1710_04751_gb300 import net
    peak, kind = measured_peak_tflops()
    gen = torch.Generator(device="cuda").manual_seed(0)

    def back_to_back(call, reps):
        """Seconds per call: `reps` calls queued back to back between two events (the host
        work of a call -- tensor-map encoding, argument checks -- overlaps the kernel of the
        call before it), best of 3."""
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        call()
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            e0.record(st)
            for _ in range(reps):
                call()
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) * 1e-3 / reps)
        return best

    def gemm_rate(M, N, K, mode, splits=1, reps=10):
        A = torch.randn((M, K), device="cuda", generator=gen).to(torch.bfloat16)
        B = torch.randn((N, K), device="cuda", generator=gen).to(torch.bfloat16)
        C = torch.zeros((M, N), device="cuda",
                        dtype=torch.bfloat16 if mode == net.GEMM_BF16 else torch.float32)
        net.gemm_bf16(A, B, C, mode, splits=splits)
        best = back_to_back(lambda: net.gemm_bf16(A, B, C, mode, splits=splits), reps)
        tf = 2.0 * M * N * K / best / 1e12
        return {"M": M, "N": N, "K": K, "ms": round(best * 1e3, 4), "tflops": round(tf, 1),
                "frac": round(tf / peak, 4)}

    def wgrad_rate(B, n, cin, cout, splits, reps=10):
        """The implicit weight gradient (lbm_nn_conv3d_wgrad_bf16), scratch allocated once."""
        M = B * n ** 3
        Kp = (27 * cin + 63) // 64 * 64
        X = torch.randn((B, n ** 3, cin), device="cuda", generator=gen).to(torch.bfloat16)
        dZ = (torch.randn((M, cout), device="cuda", generator=gen) / 64).to(torch.bfloat16)
        dWT = torch.zeros((Kp, cout), device="cuda")
        ws = torch.empty(splits * Kp * cout, dtype=torch.float32, device="cuda")
        L = net._lib()

        def call():
            net._check(L.lbm_nn_conv3d_wgrad_bf16(X.data_ptr(), B, n, cin, dZ.data_ptr(), cout, Kp,
                                                  ws.data_ptr(), ws.numel(), splits, dWT.data_ptr(),
                                                  net._stream(dWT)))
        best = back_to_back(call, reps)
        tf = 2.0 * M * 27 * cin * cout / best / 1e12
        return {"M": 27 * cin, "N": cout, "K": M, "ms": round(best * 1e3, 4), "tflops": round(tf, 1),
                "frac": round(tf / peak, 4)}

    def conv_rate(B, n, cin, cout, mode, reps=10):
        """The implicit-GEMM convolution (no im2col matrix): time, TFLOP/s and the bytes it
        must move at least (input and output once)."""
        X = torch.randn((B, n ** 3, cin), device="cuda", generator=gen).to(torch.bfloat16)
        ldw = (27 * cin + 63) // 64 * 64
        W = (0.05 * torch.randn((cout, ldw), device="cuda", generator=gen)).to(torch.bfloat16)
        bias = torch.zeros(cout, device="cuda")
        out = torch.empty((B * n ** 3, cout), device="cuda",
                          dtype=torch.bfloat16 if mode == net.CONV_BIAS_RELU_BF16 else torch.float32)
        net.conv3d_bf16(X, n, W, out, mode=mode, bias=bias)
        best = back_to_back(lambda: net.conv3d_bf16(X, n, W, out, mode=mode, bias=bias), reps)
        tf = 2.0 * B * n ** 3 * 27 * cin * cout / best / 1e12
        nbytes = B * n ** 3 * (2 * cin + out.element_size() * cout) + cout * ldw * 2
        return {"B": B, "n": n, "cin": cin, "cout": cout, "ms": round(best * 1e3, 4),
                "tflops": round(tf, 1), "frac": round(tf / peak, 4),
                "min_bytes": nbytes, "GB_per_s_of_min_bytes": round(nbytes / best / 1e9, 1)}

    out = {
        "peak_tflops": peak, "peak_kind": kind,
        "gemm_large": gemm_rate(65536, 256, 8192, net.GEMM_F32),
        # the network's layer 9 at 64^3, batch 2 (96 -> 32 channels): the forward pass and
        # the input gradient and the weight gradient as implicit GEMMs (the weight gradient
        # split 64 ways over the voxels, its x-shifted transposes included)
        "conv_fwd_L9": conv_rate(2, 64, 96, 32, net.CONV_BIAS_RELU_BF16),
        "conv_dgrad_L9": conv_rate(2, 64, 32, 96, net.CONV_F32),
        "conv_wgrad_L9": wgrad_rate(2, 64, 96, 32, 64),
    }
    for B in (2, 4):
        netw = net.Net(n=64, max_batch=B, seed=1)
        t = torch.randn((B, 64 ** 3, 4), device="cuda", generator=gen) * 0.3
        sc = [[0.1, 0.2]] * B
        netw.train_step(sc, t)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(5):
            netw.train_step(sc, t)
        torch.cuda.synchronize()
        ts = (time.perf_counter() - t0) / 5
        t0 = time.perf_counter()
        for _ in range(5):
            netw.forward(sc)
        torch.cuda.synchronize()
        tf = (time.perf_counter() - t0) / 5
        out[f"batch{B}"] = {"train_step_ms": round(ts * 1e3, 2), "forward_ms": round(tf * 1e3, 2)}
        out["params"] = netw.param_count
        netw.close()
    return out


def cpu_model():
    """The host CPU's model name (lscpu; /proc/cpuinfo as a fallback)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_leg(oracle, n, Ra, steps, threads, q=15):
    """One timed oracle run of the cavity at n^3 from its seeded initial state."""
    p = oracle.Problem.cavity(n, Ra, Pr=PR, Ma=U0 * math.sqrt(3.0), q_g=q)
    F, G = p.init(seed=1, noise_amp=1e-6)
    oracle.set_num_threads(threads)
    F, G = p.step(F, G)  # first touch / page-in outside the timing
    t0 = time.perf_counter()
    p.run(F, G, steps)
    dt = time.perf_counter() - t0
    return {"grid": n, "Ra": Ra, "steps": steps, "threads": threads,
            "seconds": round(dt, 3), "mlups": round(n ** 3 * steps / dt / 1e6, 3)}


def cpu_baseline():
    """The FP64 oracle, as it stands, on the host cores: the 32^3 Ra = 1e3 cavity for
    300 steps and the 64^3 one for 50 steps, each single-threaded and on every core, and
    the bench's own workload (128^3, Ra = 1e5) for 3 steps on every core.  The line's
    value is the 128^3 figure (the same workload as the GPU line)."""
    import oracle
    cores = os.cpu_count() or 1
    legs = []
    for n, Ra, steps in ((32, 1e3, 300), (64, 1e3, 50)):
        for threads in (1, cores):
            legs.append(_oracle_leg(oracle, n, Ra, steps, threads))
    main = _oracle_leg(oracle, N_GRID, RA, 3, cores)
    oracle.set_num_threads(cores)
    return {"value": main["mlups"], "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": cores,
            "sample": f"{N_GRID}^3 cavity Ra=1e5, D3Q15+D3Q15, 3 FP64 steps on {cores} threads",
            "legs": legs}


def gpu_arm(args):
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = init_dist(world, "nccl")
    import paper_1710_04751_gb300 as lbm
    lbm.load()

    peak, peak_kind = measured_peak_gbs()
    clocks = None if args.no_clocks else ClockSampler(local)
    main = run_variant(lbm, 15, args.steps, args.warmup, dist, device, clocks)
    variant = run_variant(lbm, 7, args.steps, args.warmup, dist, device, None)
    half_steps = max(1, args.steps // 4)
    sixteen = {}
    for name, prec, tname in (("FP16_DEV", lbm.FP16_DEV, "__half"), ("BF16_DEV", lbm.BF16_DEV, "__nv_bfloat16")):
        for q in (15, 7):
            sixteen[(name, q)] = (tname, run_variant(lbm, q, half_steps, args.warmup, dist, device,
                                                     None, precision=prec))

    # the same cavity at 256^3 (16.8 M nodes), FP32 and FP16, a short run of each
    big_steps = max(1, min(1000, args.steps // 20))
    big = {name: (tname, sb, run_variant(lbm, 15, big_steps, 20, dist, device, None,
                                         precision=prec, n=2 * N_GRID))
           for name, prec, tname, sb in (("FP32", lbm.FP32, "float", 4),
                                         ("FP16_DEV", lbm.FP16_DEV, "__half", 2))}

    def roof(res, q, storage_bytes=4, tname="float", traffic=None, n=N_GRID):
        bpn = bytes_per_node(q, storage_bytes)
        achieved = bpn * n ** 3 / res["t_kernel"] / 1e9
        return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "traffic_unit": "bytes per launch (ncu)" if traffic is not None else None,
                "peak_kind": peak_kind,
                # the 16-bit forms take the two-node pair kernel when nx is even
                "kernel": (f"step_pair_kernel<{tname},{q}>" if storage_bytes == 2 and n % 2 == 0
                           else f"step_cavity_kernel<{tname},{q}>"),
                "bytes_per_node": bpn, "kernel_ms": round(res["t_kernel"] * 1e3, 4)}

    total_lups = sum_over_ranks(dist, N_GRID ** 3 * args.steps, device)
    value = total_lups / main["elapsed"] / 1e6
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(main["elapsed"] / args.steps * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic: cavity at rest, T = seeded uniform noise +-1e-6",
        "config": {
            "workload": "differentially heated cubic cavity 128^3, Ra=1e5, Pr=0.71, U0=0.05, "
                        "D3Q15 flow + D3Q15 thermal, FP32, to-steady run",
            "grid": [N_GRID] * 3, "Ra": RA, "Pr": PR, "lattice": "D3Q15+D3Q15",
            "residual_interval": RESIDUAL_INTERVAL,
            "l2": "inputs larger than L2: A/B state 503 MB > 129 MB",
            "parallelism": f"replicas{world}" if world > 1 else "single",
        },
        "roofline": roof(main, 15, traffic=args.traffic.get(15)),
        "clocks": main["clocks"],
        "gpu_launches": main["launches"],
        "variants": {
            "D3Q15+D3Q7": {"value": round(sum_over_ranks(dist, N_GRID ** 3 * args.steps, device)
                                          / variant["elapsed"] / 1e6, 1),
                           "unit": "MLUPS", "ms_per_step": round(variant["elapsed"] / args.steps * 1e3, 5),
                           "roofline": roof(variant, 7, traffic=args.traffic.get(7))},
            **{f"D3Q15+D3Q{q} {name}": {
                "value": round(sum_over_ranks(dist, N_GRID ** 3 * half_steps, device)
                               / res["elapsed"] / 1e6, 1),
                "unit": "MLUPS", "steps": half_steps,
                "ms_per_step": round(res["elapsed"] / half_steps * 1e3, 5),
                "roofline": roof(res, q, 2, tname)}
               for (name, q), (tname, res) in sixteen.items()},
            **{f"256^3 D3Q15+D3Q15 {name}": {
                "value": round(sum_over_ranks(dist, (2 * N_GRID) ** 3 * big_steps, device)
                               / res["elapsed"] / 1e6, 1),
                "unit": "MLUPS", "steps": big_steps,
                "ms_per_step": round(res["elapsed"] / big_steps * 1e3, 5),
                "roofline": roof(res, 15, sb, tname, n=2 * N_GRID)}
               for name, (tname, sb, res) in big.items()},
        },
        "state_after": {"steps": args.warmup + args.steps, "Nu_hot": main["nu"]["hot_wall_mean"],
                        "residual_per_100": main["residual"]},
    }
    if not args.no_steady:
        tts15 = time_to_steady(lbm, 15, args.steady_max_steps)
        line["time_to_steady"] = {
            "D3Q15+D3Q15": tts15,
            "D3Q15+D3Q7": time_to_steady(lbm, 7, args.steady_max_steps),
        }
        if tts15["converged"]:
            line["time_to_steady"]["D3Q15+D3Q15 16-bit, FP32's step count"] = \
                time_to_steady_16bit(lbm, 15, tts15)
    if not args.no_batch:
        line["batch"] = batch_variant(lbm, args.batch_steps, RESIDUAL_INTERVAL, peak,
                                      args.batch_converge_steps)
    if not args.no_slabs:
        line["slabs"] = slab_variant(lbm, max(RESIDUAL_INTERVAL, args.steps // 10 // RESIDUAL_INTERVAL
                                          * RESIDUAL_INTERVAL), args.warmup, device,
                                     main["elapsed"] / args.steps * 1e3)
    if not args.no_net:
        line["net"] = net_variant()
    if args.warmstart:
        from paper_1710_04751_gb300 import warmstart
        res, netw = warmstart.experiment(count_train=args.ws_train, count_test=args.ws_test,
                                         count_big=args.ws_big, epochs=args.ws_epochs)
        line["warmstart"] = {"train": res["train"], "test": res["test"]["summary"],
                             "big": res["big"]["summary"] if res["big"] else None}
        netw.close()
    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_variant(lbm, 15, args.e2e_reps, device)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def reference_arm(args):
    """The reference arm is the FP64 CPU oracle on the host's cores (rank 0 only).  Each
    bench step is one oracle time step of a bounded sample of the workload: a
    128 x 128 x nz slab of the same cavity (same Ra, Pr, U0 and wall rules), nz chosen
    so that warm-up plus timed steps take about --ref-budget seconds."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    par = oracle.physical_parameters(N_GRID, RA, PR, U0 * math.sqrt(3.0))

    def slab(nz):
        return oracle.Problem(N_GRID, N_GRID, nz, q_g=15, omega_nu=par["omega_nu"],
                              omega_phi=par["omega_phi"], gbeta=par["gbeta"], U0=par["U0"])

    cal = slab(8)
    F, G = cal.init(seed=1, noise_amp=1e-6)
    t0 = time.perf_counter()
    cal.step(F, G)
    rate = cal.ncell / max(time.perf_counter() - t0, 1e-6)  # node updates per second
    per_step = args.ref_budget / max(1, args.steps + args.warmup)
    nz = int(max(1, min(N_GRID, per_step * rate / (N_GRID * N_GRID))))
    p = slab(nz)
    F, G = p.init(seed=1, noise_amp=1e-6)
    for _ in range(args.warmup):
        F, G = p.step(F, G)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        F, G = p.step(F, G)
    dt = time.perf_counter() - t0
    value = p.ncell * args.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle time step of a {N_GRID}x{N_GRID}x{nz} slab of the "
              f"128^3 Ra=1e5 cavity ({p.ncell} nodes); {args.steps} timed after {args.warmup}")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "differentially heated cubic cavity 128^3, Ra=1e5, Pr=0.71, U0=0.05, "
                               "D3Q15 flow + D3Q15 thermal (FP64 CPU oracle, bounded sample)",
                   "grid": [N_GRID] * 3, "Ra": RA, "Pr": PR, "lattice": "D3Q15+D3Q15"},
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-reps", type=int, default=20)
    ap.add_argument("--no-steady", action="store_true",
                    help="skip the run of both variants from rest to steady state")
    ap.add_argument("--steady-max-steps", type=int, default=400_000)
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-cavity batched form")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--no-net", action="store_true", help="skip the warm-start network timings")
    ap.add_argument("--no-slabs", action="store_true", help="skip the z-slab decomposition timings")
    ap.add_argument("--no-clocks", action="store_true",
                    help="no clock sampling (and none of its load steps around the timed region)")
    ap.add_argument("--warmstart", action="store_true",
                    help="also run the learned warm start end to end (about 15 minutes)")
    ap.add_argument("--ws-train", type=int, default=400)
    ap.add_argument("--ws-test", type=int, default=50)
    ap.add_argument("--ws-big", type=int, default=8)
    ap.add_argument("--ws-epochs", type=int, default=60)
    ap.add_argument("--batch-converge-steps", type=int, default=0,
                    help="also run the 64 cavities from rest to their own convergence (max steps)")
    ap.add_argument("--ref-budget", type=float, default=90.0,
                    help="seconds the reference arm spends on warm-up + timed steps")
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch of step_cavity_kernel<float,15>
    # at 128^3, from one ncu capture; to be retaken whenever that kernel changes
    ap.add_argument("--traffic-q15", type=float, default=455.7e6,
                    help="ncu DRAM bytes per launch of the FP32 D3Q15 step kernel at 128^3")
    ap.add_argument("--traffic-q7", type=float, default=None)
    args = ap.parse_args(argv)
    if args.impl == "reference":
        args.steps = 20 if args.steps is None else args.steps
        args.warmup = 3 if args.warmup is None else args.warmup
        reference_arm(args)
        return
    args.steps = 20000 if args.steps is None else args.steps
    args.warmup = 300 if args.warmup is None else args.warmup
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    args.traffic = {15: args.traffic_q15, 7: args.traffic_q7}
    gpu_arm(args)


if __name__ == "__main__":
    main()
