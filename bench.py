#!/usr/bin/env python
"""Benchmark of the GB300 Fourier-Galerkin Boltzmann-Nordheim operator.

Workload (one "step" = one classical RK4 step of the whole hot path for every request
on the GPU): the 2-D classical + bosonic pair on Maxwell molecules, N = 32 modes per
dimension, R = 6, T = (3 + sqrt 2) R / 2, dt = 0.005 --
  * eps = 0 on the BKW datum at t0 = 1,
  * eps = +1 on a Gaussian of mass 5 and temperature 0.5,
in mixed precision (FP32 bulk sums with FP64 tables, transforms, accumulation of Q^,
moments and state); the same pair in FP64 is timed beside it.

Metric: Lemma terms per second ("mode-pairs/s"): each evaluation of Q_eps counts the
quadratic terms of the Lemma (pairs k+l = n in I_N) plus, when eps != 0, its cubic terms
(triples k+l+m = n), i.e. C2 = (3N^2/4)^d and C3 = (2(N^3-N)/3)^d; four evaluations per
RK4 step.  Multi-GPU runs are replicas (every rank steps its own pair; no collective on the
data path; weak scaling).

--impl reference times the FP64 CPU oracle (the reference arm of this project) on a bounded
sample of the same workload and reports the same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Q_ε mode-pairs/s & solves/s, mixed vs FP64 same GB300; p50/p99 solve latency"
UNIT = "mode-pairs/s"
N_MODES, R_TRUNC, DT = 32, 6.0, 0.005
T_END = {"bkw": 5.0 - 1.0, "boson": 5.0}   # integration spans of the two solves
L2_FLUSH_BYTES = 256 << 20
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP64_PEAK_TF = 1.25   # nominal dense FP64 of one GB300


def lemma_terms(d: int, N: int, cubic: bool) -> float:
    c2 = (0.75 * N * N) ** d
    c3 = (2.0 * (N ** 3 - N) / 3.0) ** d
    return c2 + (c3 if cubic else 0.0)


def lemma_terms_box(N: int, lo: int, cnt: int, cubic: bool) -> float:
    """Lemma terms of the outputs n in the box [lo, lo+cnt)^2 (per-dimension counts multiply)."""
    I = np.arange(-N // 2, N // 2)
    q1 = np.array([np.sum((n - I >= -N // 2) & (n - I < N // 2)) for n in range(lo, lo + cnt)], float)
    kl = (I[:, None] + I[None, :]).ravel()
    c1 = np.array([np.sum((n - kl >= -N // 2) & (n - kl < N // 2)) for n in range(lo, lo + cnt)], float)
    return float(q1.sum() ** 2 + (c1.sum() ** 2 if cubic else 0.0))


def reduce_max_over_ranks(x: float, ws: int) -> float:
    """Max of a per-rank float over all ranks (gloo all-reduce; identity for one rank)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, ws: int) -> float:
    """Weak-scaling throughput: the units all ranks processed divided by the slowest rank's time."""
    return ws * units_per_rank / seconds_max


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def clocks_sampler_start(path: str):
    q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        fh = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50"],
                             stdout=fh, stderr=subprocess.DEVNULL)
        time.sleep(0.5)   # let the sampler come up before the timed region
        return p, fh
    except Exception:
        return None, None


def clocks_sampler_stop(p, fh, path: str, gpu: int, window):
    """Median SM clock and throttle reasons from the samples taken inside `window`
    (wall-clock seconds since the epoch); falls back to every sample of the run."""
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    fh.close()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    rows = []
    for line in open(path):
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 10 or not parts[1].isdigit() or int(parts[1]) != gpu:
            continue
        try:
            ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
            frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
            rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[6:10]))
        except (ValueError, IndexError):
            continue
    if not rows:
        return None
    inside = [r for r in rows if window[0] - 0.05 <= r[0] <= window[1] + 0.05]
    used = inside if inside else rows
    reasons = sorted({n for r in used for n, flag in zip(names, r[3]) if flag.lower() == "active"})
    return {"sm_mhz": float(np.median([r[1] for r in used])), "sm_max_mhz": float(max(r[2] for r in used)),
            "reasons": reasons, "samples": len(used), "window": "timed region" if inside else "whole run"}


def source_sha(path: str) -> str:
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per launch of the fused kernel from the committed ncu summary, if the
    kernel source is unchanged since it was captured; else None."""
    src = os.path.join(ROOT, "paper_2110_13735_gb300", "csrc", "bn_fused2d_mixed.cu")
    rec = os.path.join(ROOT, "profiles", "mixed2d_traffic.json")
    if not os.path.exists(rec):
        return None
    try:
        data = json.load(open(rec))
        if data.get("kernel_sha") == source_sha(src):
            return float(data["dram_bytes_per_launch"])
    except Exception:
        return None
    return None


def workload_config(ws: int) -> dict:
    """The `config` of both arms' JSON lines (the same workload)."""
    return {"workload": "2-D Maxwell molecules N=32 R=6 T=(3+sqrt2)R/2: BKW eps=0 (t0=1) + Gaussian "
                        "(mass 5, T 0.5) eps=+1, RK4 dt=0.005, mixed precision",
            "d": 2, "N": N_MODES, "requests_per_gpu": 2, "parallelism": f"replicas x{ws}",
            "l2": "flushed between timed steps (256 MiB write, outside the step events)"}


def make_pair(bn, I, precision, stream, mixed_rw=0):
    T = I.box_half_width(R_TRUNC)
    bkw = bn.Solver(2, N_MODES, T, R_TRUNC, bn.MAXWELL, 0.0, stream=stream, precision=precision, mixed_rw=mixed_rw)
    bos = bn.Solver(2, N_MODES, T, R_TRUNC, bn.MAXWELL, 1.0, stream=stream, precision=precision, mixed_rw=mixed_rw)
    f_bkw = I.config1_bkw_f0(N_MODES, R_TRUNC)
    f_bos = I.config1_boson_f0(N_MODES, R_TRUNC)
    bkw.set_state(f_bkw)
    bos.set_state(f_bos)
    return [bkw, bos], [f_bkw, f_bos]


def fma_peaks(bn, stream):
    """Measured FMA rates of this GPU (FP32, paired FP32, FP64) with the SM clock sampled around
    them: the roofline denominators of the operator kernels."""
    clk = os.path.join(tempfile.gettempdir(), f"bn_bench_peak_clocks_{os.getpid()}.csv")
    p, fh = clocks_sampler_start(clk)
    t0 = time.time()
    res = {}
    for kind, name in ((0, "fp32"), (1, "fp32x2"), (2, "fp64")):
        best = 0.0
        for _ in range(2):
            best = max(best, bn.measure_fma_peak(kind, stream)[0])
        res[name] = best
    clocks = clocks_sampler_stop(p, fh, clk, 0, (t0, time.time()))
    res["unit"] = "TFLOP/s"
    res["sm_mhz"] = clocks["sm_mhz"] if clocks else None
    res["how"] = ("4 CTAs x 256 threads per SM, 8 independent FMA chains per thread, fastest of 3 timed launches "
                  "(CUDA events)")
    return res


def leg_3d(bn, I, which: str, steps: int, peak_fp32: float, **solver_opts):
    """A 3-D configuration in mixed precision with FP64 moments and the conservation projection:
    'config2' = hard spheres N=32, eps=-1, two Gaussians (variance 0.8, centres +-(1.5,0,0), max 0.9),
    RK4 dt=0.01; 'config4' = hard spheres N=48, eps=+1, Gaussian of mass 8 and temperature 0.4, RK4
    dt=0.002 (one evaluation only: 4e14 terms).  The kernel-mode slices are recomputed from the
    quadrature factors at every evaluation.  Times RK4 steps (config2) or evaluations (config4) with
    CUDA events on the solver's stream, the phases of every evaluation with the library's events.
    `solver_opts` (e.g. beta_budget_mb, pair_weights) go to the solver: profiling runs use them to
    keep the device memory of a capture small."""
    import torch
    N, eps, dt, f0 = (32, -1.0, 0.01, I.config2_f0(32, R_TRUNC)) if which == "config2" else \
        (48, 1.0, 0.002, I.config4_f0(48, R_TRUNC))
    T = I.box_half_width(R_TRUNC)
    stream = torch.cuda.Stream()
    t_create = time.perf_counter()
    s = bn.Solver(3, N, T, R_TRUNC, bn.HARD_SPHERE, eps, stream=stream, precision=bn.MIXED, conserve=1,
                  **solver_opts)
    t_create = time.perf_counter() - t_create
    s.set_state(f0)
    s.profile_enable(True)
    wc = s.work_counts()
    terms_eval = float(wc[0] + wc[1] + wc[2])
    out = {"workload": f"3-D hard spheres N={N}, eps={eps:+g}, mixed precision, conservation projection, "
                       f"RK4 dt={dt}", "create_s": t_create}
    ms = []
    if which == "config2":
        s.step_rk(dt, 1)   # warm-up: captures the step graph
        s.profile_nd()
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.step_rk(dt, 1)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        evals = 4 * steps
        ph = s.profile_nd()
        out.update({"steps": steps, "ms_per_step": float(np.mean(ms)),
                    "value": terms_eval * evals / (np.sum(ms) * 1e-3), "unit": UNIT})
    else:
        s.eval_collision()   # warm-up evaluation is the same size as the timed one: time one only
        s.profile_nd()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.eval_collision()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        evals = 1
        ph = s.profile_nd()
        out.update({"evaluations": 1, "ms_per_eval": ms[0], "value": terms_eval / (ms[0] * 1e-3), "unit": UNIT})
    m = s.moments()
    s.close()
    n_ev = max(1.0, ph["evals"])
    sweep_ms = ph["sweep_ms"] / n_ev
    achieved = 4.0 * ph["terms"] / (sweep_ms * 1e-3) / 1e12 if sweep_ms > 0 else None
    out["phases_ms_per_eval"] = {k: ph[k] / n_ev for k in ("pair_ms", "beta_ms", "sweep_ms", "tail_ms")}
    out["rounds"], out["ctas"] = int(ph["rounds"]), int(ph["ctas"])
    out["terms_per_eval"] = {"quadratic": float(wc[0]), "reducible": float(wc[1]), "triple": float(wc[2])}
    out["roofline"] = {"bound": "alu", "kernel": "k_triple_nd<float,8> (Q_{1,q} Toeplitz sweeps)",
                       "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                       "frac": achieved / peak_fp32 if achieved else None,
                       "basis": "4 flop (2 FP32 FMA) per Q_{1,q} term / summed sweep-launch event time per evaluation",
                       "peak_basis": "measured paired-FP32 FMA rate (bn_measure_fma_peak)"}
    out["moments_after"] = {"rho": m[0], "e": m[4], "max_f": m[7], "t": m[8]}
    return out


def leg_rescale(bn, I, steps: int, peak_fp32: float):
    """The velocity-rescaling method (Sec. 3.3, forward Euler) on a 2-D Fermi-Dirac solve: N=32,
    hbar = 3 (eps = -9), Maxwell molecules, L = 4, R = S = 2 pi / (3 + sqrt 2) on the xi box, mixed
    precision, two Gaussian bumps (not an equilibrium) started off the scale (w 25 % above sqrt(T)).
    Times `steps` rescaled steps (each: one operator evaluation, the moments of Q brought to the host,
    the temperature solve, the spectral divergence and the update) against plain evaluations of the
    same operator, and `steps` steps of the second-order RK2 form (two evaluations each), all by CUDA
    events around the calls."""
    import torch
    N, L, eps = 32, 4.0, -9.0
    S = 2.0 * math.pi / (3.0 + math.sqrt(2.0))
    j = np.arange(-N // 2, N // 2) * (2.0 * L / N)
    v = np.stack(np.meshgrid(j, j, indexing="ij"), -1)

    def f0(x):
        return 0.06 * (np.exp(-np.sum((x - [0.8, 0.3]) ** 2, -1) / 0.8) +
                       0.7 * np.exp(-np.sum((x + [0.6, 0.5]) ** 2, -1) / 0.5))

    dv = (2.0 * L / N) ** 2
    f = f0(v)
    rho = f.sum() * dv
    u = (v * f[..., None]).sum((0, 1)) * dv / rho
    e = 0.5 * (np.sum((v - u) ** 2, -1) * f).sum() * dv / rho
    stream = torch.cuda.Stream()
    with bn.Solver(2, N, math.pi, S, bn.MAXWELL, eps, stream=stream, precision=bn.MIXED) as s:
        s.set_state(f)   # any state: sized for the first evaluation
        w = 1.0
        s.rescale_set(L, w, u, rho, e)
        T = s.rescale_state()["T"]
        w = 1.25 * math.sqrt(T)
        sc = math.pi * w / L
        xi = np.stack(np.meshgrid(*(2 * [np.arange(-N // 2, N // 2) * (2 * math.pi / N)]), indexing="ij"), -1)
        s.set_state(f0(u + xi / sc) / sc ** 2)
        s.rescale_set(L, w, u, rho, e)
        s.step_rescaled(0.01, 2)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_rescaled(0.01, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / steps
        st = s.rescale_state()
        e0.record(stream)
        for _ in range(steps):
            s.eval_collision_modes()
        e1.record(stream)
        torch.cuda.synchronize()
        eval_ms = e0.elapsed_time(e1) / steps
        # the second-order RK2 form from the same state (two evaluations per step)
        s.step_rescaled(0.01, 1, rk2=True)   # warm-up (allocates its buffer)
        torch.cuda.synchronize()
        e0.record(stream)
        s.step_rescaled(0.01, steps, rk2=True)
        e1.record(stream)
        torch.cuda.synchronize()
        rk2_ms = e0.elapsed_time(e1) / steps
    terms = lemma_terms(2, N, True)
    return {"workload": "2-D Fermi-Dirac (hbar = 3) N=32, velocity rescaling (forward Euler), L = 4, mixed precision",
            "steps": steps, "ms_per_step": step_ms, "ms_per_plain_evaluation": eval_ms,
            "rescaling_overhead": step_ms / eval_ms - 1.0, "rk2_ms_per_step": rk2_ms,
            "value": terms / (step_ms * 1e-3), "unit": UNIT,
            "sweep_fraction_of_peak_bound": 4.0 * (2.0 * (N ** 3 - N) / 3.0) ** 2 / (step_ms * 1e-3) / 1e12 / peak_fp32,
            "after": {"w": st["w"], "T": st["T"], "z": st["z"], "t": st["t"]}}


def leg_rescale3d(bn, steps: int):
    """The velocity-rescaling method in 3-D at 32^3: hard spheres, Fermi-Dirac (eps = -1), mixed
    precision, L = 6, R = S = 2 pi / (3 + sqrt 2) on the xi box, two Gaussian bumps (variance 0.8,
    centres +-(1.5, 0, 0), 0.45 each) started on the scale (w = sqrt(T) of their discrete moments).
    Times `steps` forward Euler steps and `steps` steps of the RK2 form (two evaluations each)
    against plain evaluations of the same operator, by CUDA events on the solver's stream."""
    import torch
    N, L, eps = 32, 6.0, -1.0
    S = 2.0 * math.pi / (3.0 + math.sqrt(2.0))
    c = np.array([1.5, 0.0, 0.0])

    def f0(x):
        return 0.45 * (np.exp(-np.sum((x - c) ** 2, -1) / 1.6) + np.exp(-np.sum((x + c) ** 2, -1) / 1.6))

    j = np.arange(-N // 2, N // 2) * (2.0 * L / N)
    v = np.stack(np.meshgrid(j, j, j, indexing="ij"), -1)
    dv = (2.0 * L / N) ** 3
    f = f0(v)
    rho = f.sum() * dv
    u = (v * f[..., None]).sum((0, 1, 2)) * dv / rho
    e = 0.5 * (np.sum((v - u) ** 2, -1) * f).sum() * dv / rho
    T, z = bn.equilibrium_temperature(3, eps, rho, e)
    w = math.sqrt(T)
    sc = math.pi * w / L
    xi1 = np.arange(-N // 2, N // 2) * (2.0 * math.pi / N)
    xi = np.stack(np.meshgrid(xi1, xi1, xi1, indexing="ij"), -1)
    stream = torch.cuda.Stream()
    t_create = time.perf_counter()
    with bn.Solver(3, N, math.pi, S, bn.HARD_SPHERE, eps, stream=stream, precision=bn.MIXED) as s:
        t_create = time.perf_counter() - t_create
        s.set_state(f0(u + xi / sc) / sc ** 3)
        s.rescale_set(L, w, u, rho, e)
        s.step_rescaled(0.01, 1)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.step_rescaled(0.01, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        euler_ms = e0.elapsed_time(e1) / steps
        e0.record(stream)
        s.step_rescaled(0.01, steps, rk2=True)
        e1.record(stream)
        torch.cuda.synchronize()
        rk2_ms = e0.elapsed_time(e1) / steps
        e0.record(stream)
        for _ in range(steps):
            s.eval_collision_modes()
        e1.record(stream)
        torch.cuda.synchronize()
        eval_ms = e0.elapsed_time(e1) / steps
        st = s.rescale_state()
    return {"workload": "3-D hard spheres N=32, Fermi-Dirac eps=-1, velocity rescaling, L = 6, mixed precision",
            "create_s": t_create, "steps": steps, "x": abs(eps) * rho * (3.0 / (4.0 * math.pi * e)) ** 1.5,
            "ms_per_euler_step": euler_ms, "ms_per_rk2_step": rk2_ms, "ms_per_plain_evaluation": eval_ms,
            "rescaling_overhead": euler_ms / eval_ms - 1.0,
            "before": {"w": w, "T": T, "z": z}, "after": {"w": st["w"], "T": st["T"], "z": st["z"], "t": st["t"]}}

def leg_2d64(bn, I, evals: int, peak_fp32: float):
    """The largest serving size alone: 2-D Maxwell molecules N=64, R=6, the Gaussian of mass 5 and
    temperature 0.5 with eps=+1, mixed precision; `evals` evaluations after two warm-up ones, timed
    with CUDA events on the solver's stream."""
    import torch
    N = 64
    T = I.box_half_width(R_TRUNC)
    stream = torch.cuda.Stream()
    with bn.Solver(2, N, T, R_TRUNC, bn.MAXWELL, 1.0, stream=stream, precision=bn.MIXED) as s:
        s.set_state(I.config1_boson_f0(N, R_TRUNC))
        for _ in range(2):
            s.eval_collision()
        ms = []
        for _ in range(evals):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s.eval_collision_modes()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    terms = (2.0 * (N ** 3 - N) / 3.0) ** 2
    t = float(np.median(ms))
    return {"workload": "2-D Maxwell molecules N=64, Gaussian (mass 5, temperature 0.5), eps=+1, mixed precision",
            "evaluations": evals, "ms_per_eval_median": t,
            "achieved_tflops": 4.0 * terms / (t * 1e-3) / 1e12,
            "frac": 4.0 * terms / (t * 1e-3) / 1e12 / peak_fp32,
            "basis": "4 flop per Q_{1,q} term / whole-evaluation event time (transforms and partial sums included)"}


def run_leg_only(args):
    """One leg alone (`--only config2|config4|2d64|rescale|rescale3d`), printed as one JSON line: the
    profiling runs' command, with the 3-D solver's slice budget and pair-weight mode set from the
    command line."""
    import torch
    torch.cuda.set_device(0)
    from paper_2110_13735_gb300 import build as BUILD
    BUILD.build()
    from paper_2110_13735_gb300 import bn
    from paper_2110_13735_gb300 import inputs as I
    bn.load()
    if args.only == "rescale3d":
        print(json.dumps({"leg": args.only, **leg_rescale3d(bn, max(1, args.leg3d_steps))}))
        return
    if args.only in ("2d64", "rescale"):
        peak = bn.measure_fma_peak(1, None)[0]
        leg = leg_2d64(bn, I, max(3, args.steps), peak) if args.only == "2d64" else \
            leg_rescale(bn, I, max(3, args.leg_rescale), peak)
        print(json.dumps({"leg": args.only, **leg}))
        return
    opts = {}
    if args.beta_budget_mb > 0:
        opts["beta_budget_mb"] = args.beta_budget_mb
    if args.pair_weights:
        opts["pair_weights"] = 1
    peak = bn.measure_fma_peak(1, None)[0]
    leg = leg_3d(bn, I, args.only, max(1, args.leg3d_steps), peak, **opts)
    print(json.dumps({"leg": args.only, "solver_options": opts, **leg}))


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2110_13735_gb300 import build as BUILD
    if rank == 0 or ws == 1:
        BUILD.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_2110_13735_gb300 import bn
    from paper_2110_13735_gb300 import inputs as I
    bn.load()
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    peaks = fma_peaks(bn, stream)

    terms_step = 4.0 * (lemma_terms(2, N_MODES, False) + lemma_terms(2, N_MODES, True))

    def timed(solvers, steps, warmup, profile=False):
        dts = [DT] * len(solvers)
        for _ in range(warmup):
            bn.step_rk_batch(solvers, dts, 1)
        if profile:
            # the shared step graph stamps every fused launch (all requests of one evaluation)
            solvers[0].profile_enable(True)
            bn.step_rk_batch(solvers, dts, 1)   # recapture with the stamps
            solvers[0].profile_read()
        launches0 = sum(s.kernel_launches() for s in solvers)
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        evs = []
        t_wall0 = time.time()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bn.step_rk_batch(solvers, dts, 1)
            e1.record(stream)
            evs.append((e0, e1))
        torch.cuda.synchronize()
        t_wall1 = time.time()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        launches = sum(s.kernel_launches() for s in solvers) - launches0
        prof = None
        if profile:
            prof = solvers[0].profile_read()
            solvers[0].profile_enable(False)
        return ms, launches, prof, (t_wall0, t_wall1)

    # ---- mixed precision (the headline)
    solvers, f0 = make_pair(bn, I, bn.MIXED, stream, args.mixed_rw)
    clk_path = os.path.join(tempfile.gettempdir(), f"bn_bench_clocks_rank{rank}_{os.getpid()}.csv")
    p, fh = clocks_sampler_start(clk_path)
    ms, launches, prof, window = timed(solvers, args.steps, args.warmup, profile=True)
    clocks = clocks_sampler_stop(p, fh, clk_path, local, window)
    total_ms = reduce_max_over_ranks(float(np.sum(ms)), ws)
    value = whole_job_rate(terms_step * args.steps, total_ms * 1e-3, ws)
    ms_per_step = total_ms / args.steps

    # ---- end to end through the public API with host buffers (copies inside the timed region)
    # inputs and results in pinned host memory (page-locked, as a serving front end would keep them)
    h_in = [torch.empty(f.size, dtype=torch.float64, pin_memory=True).numpy() for f in f0]
    for h, f in zip(h_in, f0):
        h[:] = f.reshape(-1)
    h_out = [torch.empty(h.size, dtype=torch.float64, pin_memory=True).numpy() for h in h_in]
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s, h in zip(solvers, h_in):
            s.set_state(h)
        bn.step_rk_batch(solvers, [DT] * 2, 1)
        for s, o in zip(solvers, h_out):
            s.get_state(out=o)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = ws * terms_step * e2e_steps / e2e_s
    bytes_io = sum(h.nbytes for h in h_in)

    # ---- dominant kernel: live timing of the fused operator kernel inside the timed steps.  One
    # launch per evaluation serves both requests (the shared step graph); its algorithmic work is
    # the Q_{1,q} triple sum of the eps=+1 request, 4 flop (2 FFMA) per term.  The eps=0 request's
    # quadratic terms (0.1% of the work) are not counted.
    flops_launch = 4.0 * (2.0 * (N_MODES ** 3 - N_MODES) / 3.0) ** 2
    peak = peaks["fp32x2"]
    kcfg = solvers[1].kernel_config()
    kern_ms, basis = None, None
    if prof and prof[3] > 0 and prof[2] > 0:
        kern_ms, basis = prof[2] / prof[3], "kernel %globaltimer span (first CTA start to last CTA end) of every launch in the timed steps"
    achieved = flops_launch / (kern_ms * 1e-3) / 1e12 if kern_ms else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if achieved else None,
                "traffic": recorded_traffic(),
                "kernel": f"k_mixed2d_batch<{kcfg[0]}> (whole 2-D operator, both requests of one evaluation; "
                          f"{kcfg[0]} outputs/thread chosen by the autotuner, {kcfg[1]} CTAs per request)",
                "launches_timed": int(prof[3]) if prof else 0, "ms_per_launch": kern_ms,
                "timing": basis,
                "peak_basis": f"measured paired-FP32 FMA rate of this GPU (bn_measure_fma_peak) at "
                              f"{peaks['sm_mhz']} MHz; unit counts at the maximum clock give "
                              f"{SM_COUNT * FP32_LANES * 2.0 * SM_MAX_MHZ * 1e6 / 1e12:.1f}"}
    if clocks and achieved and peaks.get("sm_mhz"):
        roofline["frac_at_median_clock"] = achieved / (peak * clocks["sm_mhz"] / peaks["sm_mhz"])
    for s in solvers:
        s.close()

    # ---- FP64 beside it (fewer steps)
    fp64, ms64_step = None, None
    if not args.no_fp64:
        solvers64, _ = make_pair(bn, I, bn.FP64, stream)
        k64 = max(3, args.steps // 4)
        ms64, _, prof64, _ = timed(solvers64, k64, min(args.warmup, 3), profile=True)
        for s in solvers64:
            s.close()
        ms64_step = float(np.mean(ms64))
        fp64 = {"value": terms_step / (ms64_step * 1e-3) * ws, "unit": UNIT, "ms_per_step": ms64_step, "steps": k64}
        if prof64 and prof64[3] > 0 and prof64[2] > 0:
            k64_ms = prof64[2] / prof64[3]
            a64 = flops_launch / (k64_ms * 1e-3) / 1e12
            fp64["roofline"] = {"bound": "alu", "kernel": "k_fused2d_batch<double,2,128> (both requests)",
                                "ms_per_launch": k64_ms, "achieved": a64, "peak": peaks["fp64"], "unit": "TFLOP/s",
                                "frac": a64 / peaks["fp64"],
                                "peak_basis": f"measured FP64 FMA rate of this GPU (bn_measure_fma_peak); "
                                              f"nominal {FP64_PEAK_TF}"}

    steps_to_end = {k: int(round(v / DT)) for k, v in T_END.items()}
    solves = {"pair_solve_s_mixed": ms_per_step * max(steps_to_end.values()) / 1e3}
    solves["solves_per_s_mixed"] = ws * 2.0 / solves["pair_solve_s_mixed"]
    if ms64_step is not None:
        solves["pair_solve_s_fp64"] = ms64_step * max(steps_to_end.values()) / 1e3
        solves["solves_per_s_fp64"] = ws * 2.0 / solves["pair_solve_s_fp64"]

    def guarded(fn, *a, **kw):
        """An extra leg: its failure is recorded in its field of the JSON line, not raised (the
        headline numbers above are already measured)."""
        try:
            return fn(*a, **kw)
        except Exception as exc:   # noqa: BLE001 -- any failure of a side leg
            return {"error": f"{type(exc).__name__}: {exc}"}

    serving = None
    if args.serving > 0 and ws == 1:   # extra legs at N=1 only (replicas would repeat them)
        Ns = tuple(int(x) for x in args.serving_ns.split(","))
        per_n = {int(a): int(b) for a, b in (x.split(":") for x in args.serving_fp64.split(","))}
        policy = {"beta_split_N": sorted(int(x) for x in args.serving_beta_split.split(",") if x),
                  "escalate_at_by_N": {int(a): float(b) for a, b in (x.split(":") for x in args.serving_escalate.split(",")
                                                                     if x)}}
        serving = guarded(serving_sample, bn, I, args.serving, 200.0, {N: per_n.get(N, 0) for N in Ns}, Ns=Ns,
                          policy=policy)

    legs = {}
    if args.leg3d_steps > 0 and ws == 1:
        legs["config2_3d_n32"] = guarded(leg_3d, bn, I, "config2", args.leg3d_steps, peaks["fp32x2"])
    if args.leg48 and ws == 1:
        legs["config4_3d_n48"] = guarded(leg_3d, bn, I, "config4", 1, peaks["fp32x2"])
    if args.leg_rescale > 0 and ws == 1:
        legs["rescaling_2d_n32"] = guarded(leg_rescale, bn, I, args.leg_rescale, peaks["fp32x2"])

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = guarded(cpu_baseline_sample, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": workload_config(ws),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": bytes_io, "d2h_bytes_per_step": bytes_io,
                    "steps": e2e_steps},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "gpu_launches": int(launches),
            "fp64": fp64,
            "solves": solves,
            "serving": serving,
            "fma_peaks": peaks,
            "legs": legs,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serving_run(bn, I, reqs, policy: dict):
    """Continuous-batching server on a seeded stream of 2-D requests fed in real time from a host
    thread (mixed precision with the per-request options of `policy`).  Returns (latencies, final
    states, wall seconds, server stats); the stats also list the requests that switched to FP64."""
    import threading
    T = I.box_half_width(6.0)
    f0s = [I.request_f0(r) for r in reqs]
    ids = [None] * len(reqs)
    # 64 slots, least estimated work first: the cheap requests pass while the N=64 ones queue (all
    # admitted at once, every request would finish in the last steps of one shared batch)
    with bn.Server(max_active=64) as srv:
        def feeder():
            t_start = time.perf_counter()
            for k, r in enumerate(reqs):
                delay = r["arrival"] - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                ids[k] = srv.submit(2, r["N"], T, r["R"], r["kernel"], r["eps"], f0s[k], r["dt"], r["t_end"],
                                    precision=bn.MIXED, **request_options(r, policy))
        t0 = time.perf_counter()
        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        srv.wait_idle(1800)
        wall = time.perf_counter() - t0
        lat, results, escalated = [], [], []
        for k, r in enumerate(reqs):
            st, res, times = srv.poll(ids[k], r["N"] ** 2)
            if st != 2:
                raise RuntimeError(f"serving request {k} ended in state {st}")
            lat.append(times[2] - times[0])
            results.append(res)
            if times[3] >= 0:
                escalated.append(k)
        stats = srv.stats()
        stats["escalated"] = escalated
    return np.array(lat), results, wall, stats


def serving_fp64_sample(reqs, per_n: dict) -> list:
    """A stratified sample of the serving mix for the FP64 batch-of-one reference: for each N,
    `per_n[N]` requests: one classical (eps = 0) request when per_n[N] >= 3, the others spread evenly
    from the least to the most saturated quantum request of that N (ordered by |eps| max f0, the
    quantity that sets the mixed-precision error)."""
    out = []
    for N, k in sorted(per_n.items()):
        if k <= 0:
            continue
        classical = [r for r in reqs if r["N"] == N and r["eps"] == 0.0]
        quantum = sorted((r for r in reqs if r["N"] == N and r["eps"] != 0.0), key=lambda r: (abs(r["eps"]) * r["fmax"], r["id"]))
        if k >= 3 and classical:
            out.append(classical[len(classical) // 2]["id"])
            k -= 1
        if quantum:
            idx = np.unique(np.linspace(0, len(quantum) - 1, k).round().astype(int))
            out += [quantum[i]["id"] for i in idx]
    return out


def request_options(r, policy: dict) -> dict:
    """Solver options of one serving request under `policy`: the kernel-mode rounding correction for
    the N in policy['beta_split_N'], and the switch to FP64 at |eps| max f >= policy['escalate_at_by_N'][N]."""
    o = {}
    if r["N"] in policy.get("beta_split_N", ()):
        o["beta_split"] = 1
    x = policy.get("escalate_at_by_N", {}).get(r["N"], 0.0)
    if x > 0:
        o["escalate_at"] = x
    return o


def serving_sample(bn, I, n_requests: int, rate: float, per_n: dict, Ns=(16, 32, 64), policy=None):
    """The serving mix (N in `Ns`, eps in {-1, 0, +1}, Maxwell molecules or hard spheres, two-Gaussian
    data, Poisson arrivals at `rate`/s, RK4 dt=0.01 to t=2) through the continuous-batching server
    in mixed precision with the per-request options of `policy` (request_options), against a
    stratified sample of the same requests solved one at a time in FP64: p50/p99 time to solution,
    solves/s, and the relative L2 difference of the final states.  The FP64 batch-of-one rate of the
    whole mix is the measured per-N solve times weighted by the mix's N counts."""
    policy = policy or {}
    reqs = I.serving_requests(n=n_requests, rate=rate, Ns=Ns, kernels=(0, 1))
    T = I.box_half_width(6.0)
    sample = serving_fp64_sample(reqs, per_n)
    t_by_n, refs = {}, {}
    for k in sample:
        r = reqs[k]
        with bn.Solver(2, r["N"], T, r["R"], r["kernel"], r["eps"], precision=bn.FP64) as s:
            s.set_state(I.request_f0(r))
            a = time.perf_counter()
            s.step_rk(r["dt"], int(round(r["t_end"] / r["dt"])))
            refs[k] = s.get_state().reshape(-1)
            t_by_n.setdefault(r["N"], []).append(time.perf_counter() - a)
    counts = {N: sum(1 for r in reqs if r["N"] == N) for N in Ns}
    fp64_mix_s = sum(counts[N] * float(np.mean(t_by_n[N])) for N in Ns if N in t_by_n)
    lat, results, wall, stats = serving_run(bn, I, reqs, policy)
    rel = {k: float(np.linalg.norm(results[k] - refs[k]) / np.linalg.norm(refs[k])) for k in sample}
    lat = np.asarray(lat)
    by_n = {}
    for N in Ns:
        sel = [i for i, r in enumerate(reqs) if r["N"] == N]
        e = [rel[k] for k in sample if reqs[k]["N"] == N]
        by_n[str(N)] = {"requests": len(sel), "escalated_to_fp64": sum(1 for k in stats["escalated"] if reqs[k]["N"] == N),
                        "p50_s": float(np.percentile(lat[sel], 50)),
                        "p99_s": float(np.percentile(lat[sel], 99)),
                        "fp64_batch_of_one_s": float(np.mean(t_by_n[N])) if N in t_by_n else None,
                        "fp64_sample": len(e), "max_rel_l2_vs_fp64": max(e) if e else None,
                        "within_1e-6": int(sum(x <= 1e-6 for x in e))}
    worst = max(sample, key=lambda k: rel[k]) if sample else None
    return {"requests": len(reqs), "arrival_rate_per_s": rate, "N": list(Ns), "kernels": ["maxwell", "hard_sphere"],
            "eps": [-1, 0, 1], "t_end": reqs[0]["t_end"], "dt": reqs[0]["dt"],
            "precision": "mixed",
            "policy": {"beta_split_N": list(policy.get("beta_split_N", ())),
                       "escalate_at_by_N": {str(k): v for k, v in policy.get("escalate_at_by_N", {}).items()}},
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "solves_per_s": len(reqs) / wall, "wall_s": wall, "max_running": stats["max_active"],
            "ticks": stats["ticks"], "escalated_to_fp64": len(stats["escalated"]),
            "fp64_batch_of_one": {"solves_per_s_mix": len(reqs) / fp64_mix_s if fp64_mix_s > 0 else None,
                                  "basis": "measured FP64 solve time per N (one request at a time) x the mix's "
                                           "N counts"},
            "fp64_sample": {"requests": len(sample), "within_1e-6": int(sum(x <= 1e-6 for x in rel.values())),
                            "max_rel_l2_vs_fp64": rel[worst] if worst is not None else None,
                            "median_rel_l2_vs_fp64": float(np.median(list(rel.values()))) if rel else None,
                            "worst": {k: reqs[worst][k] for k in ("id", "N", "eps", "kernel", "fmax", "sigma")}
                            if worst is not None else None},
            "by_N": by_n}


def host_cpu() -> dict:
    """The host CPU as lscpu names it (model, sockets x cores, threads per core)."""
    info = {}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            info[k.strip()] = v.strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": info.get("Model name") or info.get("Vendor ID"), "architecture": info.get("Architecture"),
            "cpus": info.get("CPU(s)"), "sockets": info.get("Socket(s)"), "cores_per_socket": info.get("Core(s) per socket"),
            "threads_per_core": info.get("Thread(s) per core")}


def cpu_baseline_sample(seconds: float):
    """The oracle as it stands on this host: full Lemma evaluations of the two requests at
    N=32, repeated until `seconds` of CPU time have passed, on all host threads and then, for
    a third of that time, on one thread."""
    import oracle as O
    from paper_2110_13735_gb300 import inputs as I
    T = I.box_half_width(R_TRUNC)
    ops = [(O.Operator(2, N_MODES, T, R_TRUNC, 0, 0.0), I.config1_bkw_f0(N_MODES, R_TRUNC), False),
           (O.Operator(2, N_MODES, T, R_TRUNC, 0, 1.0), I.config1_boson_f0(N_MODES, R_TRUNC), True)]
    for op, _, _ in ops:
        op.beta()

    def run(limit):
        terms, evals, t0 = 0.0, 0, time.perf_counter()
        while True:
            for op, f, cubic in ops:
                op.eval_collision(f)
                terms += lemma_terms(2, N_MODES, cubic)
                evals += 1
            if time.perf_counter() - t0 >= limit:
                break
        return terms / (time.perf_counter() - t0), evals, time.perf_counter() - t0

    threads = O.num_threads()
    value, evals, el = run(seconds)
    O.set_threads(1)
    try:
        v1, e1, el1 = run(seconds / 3.0)
    finally:
        O.set_threads(threads)
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{evals} full FP64 evaluations of Q_eps (N=32 BKW eps=0 and Gaussian eps=+1), {el:.1f} s",
            "one_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": f"{e1} evaluations, {el1:.1f} s"},
            "host": host_cpu()}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_2110_13735_gb300 import inputs as I
    T = I.box_half_width(R_TRUNC)
    op_b = O.Operator(2, N_MODES, T, R_TRUNC, 0, 1.0)
    op_c = O.Operator(2, N_MODES, T, R_TRUNC, 0, 0.0)
    g_b = op_b.dft(I.config1_boson_f0(N_MODES, R_TRUNC))
    g_c = op_c.dft(I.config1_bkw_f0(N_MODES, R_TRUNC))
    op_b.beta()
    op_c.beta()
    lo, cnt = -8, 16   # sample: the central 16x16 output modes of each request
    terms_step = lemma_terms_box(N_MODES, lo, cnt, True) + lemma_terms_box(N_MODES, lo, cnt, False)

    def step():
        op_b.collision_modes(g_b, lo, cnt)
        op_c.collision_modes(g_c, lo, cnt)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = time.perf_counter() - t0
    value = terms_step * args.steps / el
    sample = (f"per step: Lemma sums of the central 16x16 of 32x32 output modes for the Gaussian eps=+1 and "
              f"BKW eps=0 requests (FP64 oracle, {O.num_threads()} threads)")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(ws),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", type=int, default=512, help="requests of the serving mix (0 = skip)")
    ap.add_argument("--serving-ns", default="16,32,64", help="mode counts N of the serving mix")
    ap.add_argument("--serving-fp64", default="16:6,32:5,64:2",
                    help="FP64 batch-of-one reference requests per N (stratified by |eps| max f0)")
    ap.add_argument("--serving-beta-split", default="16",
                    help="mode counts N whose serving requests use the kernel-mode rounding correction (beta_split)")
    ap.add_argument("--serving-escalate", default="32:0.5",
                    help="N:x pairs: requests of that N switch to FP64 once |eps| max f >= x (others never)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 leg (profiling runs)")
    ap.add_argument("--leg3d-steps", type=int, default=1,
                    help="timed RK4 steps of the 3-D N=32 configuration (0 = skip)")
    ap.add_argument("--leg48", action="store_true", help="also time one evaluation of the 3-D N=48 configuration")
    ap.add_argument("--leg-rescale", type=int, default=20,
                    help="timed steps of the 2-D velocity-rescaling leg (0 = skip)")
    ap.add_argument("--only", choices=["config2", "config4", "2d64", "rescale", "rescale3d"],
                    help="run one leg alone and print it (profiling runs): a 3-D configuration, or the 2-D "
                         "N=64 mixed operator (--steps evaluations)")
    ap.add_argument("--beta-budget-mb", type=int, default=0,
                    help="with --only: device memory (MiB) for the kernel-mode slices of one round (0 = default)")
    ap.add_argument("--pair-weights", action="store_true",
                    help="with --only: recompute the pair weights per evaluation instead of storing them")
    ap.add_argument("--mixed-rw", type=int, default=0, choices=[0, 8, 16],
                    help="outputs per thread of the mixed kernel (0 = autotuner; profiling runs fix it)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_leg_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
