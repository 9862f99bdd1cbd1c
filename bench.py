#!/usr/bin/env python
"""Benchmark: 2D SGN RK4 steps/s on the 2048^2 Gaussian-hump workload.

Workload: h = 1 + 0.5 exp(-(x^2+y^2)), v = 0 on [-50,50)^2, 2048 x 2048 points,
dt = 1e-3, GMRES restart 20 and tolerance 1e-10 on the FP64 residual of every
solve. One step is one classic RK4 step (4 right-hand sides, each with its
GMRES solve): the whole hot path. Inputs are resident in HBM when the timed
region starts; the state and the Krylov basis (about 1.3 GB) are far larger
than L2, so no flush is needed.

The headline is ONE configuration, timed on its own: precision 2 (FP32
transforms, pointwise work and inner GMRES; double-float refinement residual
and coefficients; FP64 state), the polynomial GMRES start (guess 3), each RK4
step replayed as one CUDA graph. Beside it, the paper's method (plain FP64,
GMRES started from the last sigma) is timed the same way (`fp64_plain`), and
the host-driven loop of the headline's kernels is timed with per-launch
CUDA events for the roofline of its dominant kernel.

The LAST stdout line is one compact JSON object (a few KB). Everything else
(per-kernel tables, extra arms, ensembles, 4096^2 runs) goes to the detail
file (--detail, default bench_detail.json). Under torchrun every
rank steps its own replica (weak scaling, no collective on the data path);
value = total steps of all ranks / max time over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead: each
step is one whole oracle RK4 step of the same workload at 512^2, scaled to
2048^2 by the measured cost ratio of one oracle matvec at the two sizes.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SGN RK4 steps/s at 2048² to fixed GMRES tol: plain FP64 vs mixed+learned"
UNIT = "steps/s"
N_DEFAULT, L_DEFAULT, ALPHA, DT = 2048, 100.0, 0.5, 1e-3
# the CPU oracle's bounded sample: whole RK4 steps of the same workload on a
# coarser grid of the same box (well resolved: the hump's spectrum is below
# 1e-25 at the 512-point Nyquist wavenumber)
ORACLE_SAMPLE_N = 512

# the headline configuration: (precision, guess, graph)
HEADLINE = (2, 3, 1)
HEADLINE_PATH = ("precision 2: FP32 transforms, pointwise work and inner GMRES, FP64 state, dots and Givens, "
                 "double-float refinement residual and coefficients, every solve to the FP64 tolerance; "
                 "GMRES start: each stage's sigma from the cubic in time through the same stage of the last "
                 "4 steps; each RK4 step one CUDA graph with device-side GMRES control")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="grid points per side (default 2048)")
    ap.add_argument("--sample-n", type=int, default=ORACLE_SAMPLE_N,
                    help="grid side of the CPU oracle's sample (default 512)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None, help="steps of the end-to-end leg (default: --steps)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 arm")
    ap.add_argument("--no-prof", action="store_true", help="skip the host-loop arm with per-launch timers")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the built-in launch shapes (no sgn_autotune before the warm-up)")
    ap.add_argument("--full", action="store_true",
                    help="also run the other arms, the learned start, the 64-member ensemble and the 4096^2 "
                         "crossing solitons (detail file only)")
    ap.add_argument("--transverse", action="store_true",
                    help="also run the transverse-stability workload to t = 10 (detail file only)")
    ap.add_argument("--detail", default="bench_detail.json",
                    help="where the detailed record goes")
    return ap.parse_args(argv)


def config(n, precision_desc):
    return {"workload": f"gaussian_hump_{n}x{n}", "grid": [n, n], "box": [-L_DEFAULT / 2, L_DEFAULT / 2],
            "h0": f"1+{ALPHA}*exp(-(x^2+y^2))", "v0": "0", "dt": DT, "gmres_restart": 20, "gmres_tol": 1e-10,
            "precision": precision_desc,
            "l2": "inputs larger than L2 (state + Krylov basis, 0.9-1.3 GB resident), no flush"}


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thr = threading.Thread(target=self._read, daemon=True)
            self.thr.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    """Median SM clock under load, the maximum clock and the throttle reasons
    seen in nvidia-smi csv lines (index, sm, max sm, power, reasons...)."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        f = [x.strip() for x in ln.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for n, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(n)
    sm.sort()
    med = sm[len(sm) // 2] if sm else None
    return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, world: int) -> float:
    """Maximum of a per-rank float over all ranks (identity for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: float, seconds_local: float, world: int):
    """Whole-job units/s: all ranks' units over the slowest rank's time."""
    t = max_over_ranks(seconds_local, world)
    return world * units_per_rank / t, t


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# is now (built-in shape, radix plan 0), and the fractions of cycles it issued
# instructions and kept the FMA pipe busy (the compute view of a kernel bound
# by issue rather than by DRAM), with the summary that holds the
# command. An entry is removed when its kernel changes, and the line reports
# null when the tuned handle runs the pass in the other radix plan.
MEASURED_TRAFFIC = {
    ("ref_x", "df", 2048): {"bytes": 134.5e6 + 23.5e6, "issue": 0.70, "fma": 0.57, "source": "profiles/k_mv_x_df_gaussian2048.md"},
    ("ref_yinv", "df", 2048): {"bytes": 38.5e6 + 15.7e6, "issue": 0.57, "fma": 0.42, "source": "profiles/k_mv_x_df_gaussian2048.md"},
    ("ref_yfwd", "df", 2048): {"bytes": 84.6e6 + 8.6e6, "issue": 0.53, "fma": 0.39, "source": "profiles/k_mv_x_df_gaussian2048.md"},
    ("mv_x", "fp32", 2048): {"bytes": 67.3e6 + 22.7e6, "issue": 0.54, "fma": 0.28, "source": "profiles/k_mv_x_fp32_gaussian2048.md"},
    ("mv_yinv", "fp32", 2048): {"bytes": 16.9e6 + 0.1e6, "issue": 0.35, "fma": 0.21, "source": "profiles/k_mv_x_fp32_gaussian2048.md"},
    ("mv_yfwd", "fp32", 2048): {"bytes": 33.7e6 + 0.1e6, "issue": 0.41, "fma": 0.23, "source": "profiles/k_mv_x_fp32_gaussian2048.md"},
    ("rhs_yinv", "fp32", 2048): {"bytes": 102.2e6 + 28.0e6, "issue": 0.34, "fma": 0.18, "source": "profiles/k_ypass_fp32_gaussian2048.md"},
    ("rhs_x", "fp32", 2048): {"bytes": 100.9e6 + 7.1e6, "issue": 0.56, "fma": 0.30, "source": "profiles/k_rhs_x_fp32_gaussian2048.md"},
    ("rhs_yfwd", "fp32", 2048): {"bytes": 50.5e6 + 2.9e6, "issue": 0.26, "fma": 0.16, "source": "profiles/k_ypass_fp32_gaussian2048.md"},
}
# the (arithmetic, pass) of the tuning table each kernel class belongs to
CLASS_TUNE = {"mv_yinv": "mv_yinv", "mv_x": "mv_x", "mv_yfwd": "mv_yfwd", "rhs_yinv": "rhs_yinv", "rhs_x": "rhs_x",
              "rhs_yfwd": "rhs_yfwd", "ref_yinv": "mv_yinv", "ref_x": "mv_x", "ref_yfwd": "mv_yfwd"}

# kernel classes that are one kernel each (candidates for the roofline line)
SINGLE_KERNEL_CLASSES = ("mv_x", "mv_yinv", "mv_yfwd", "rhs_x", "rhs_yinv", "rhs_yfwd", "rk", "ref_yinv", "ref_x",
                         "ref_yfwd")


def kernel_work(cls, n, tbytes):
    """Algorithmic (flops, DRAM bytes) of one launch of a kernel class at n x n.

    tbytes: bytes per real of the pass (8 FP64 and double-float, 4 FP32); the
    RK4 state, sigma and b stay FP64 (8) in every precision. FFT flops: 5 m
    log2 m per complex transform of length m, 2.5 m log2 m per real one.
    """
    nxh = n // 2 + 1
    spec = n * nxh * 2 * tbytes       # one half spectrum of the pass's type
    spec_s = n * nxh * 2 * 8          # one FP64 half spectrum (state)
    phys = n * n * tbytes
    col = 5 * n * math.log2(n)        # one complex column FFT
    row = 2.5 * n * math.log2(n)      # one real row FFT
    if cls in ("mv_yinv", "ref_yinv"):
        return 2 * nxh * col, 3 * spec
    if cls in ("mv_x", "ref_x"):
        return n * (6 * row + 6 * n + 4 * nxh), 4 * spec + 2 * phys
    if cls in ("mv_yfwd", "ref_yfwd"):
        return 2 * nxh * col + 10 * n * nxh, 3 * spec
    if cls == "rhs_yinv":
        return 4 * nxh * col, 3 * spec_s + 4 * spec
    if cls == "rhs_x":
        return n * (8 * row + 30 * n + 6 * nxh), 4 * spec + 2 * phys + 3 * spec
    if cls == "rhs_yfwd":
        return 3 * nxh * col + 10 * n * nxh, 6 * spec
    if cls == "rk":
        # with an FP32 right-hand side the update also reads sigma_hat and the
        # stage state (the state itself at stage 1): 3.25 more FP64 spectra
        # per launch on average over the four stages
        if tbytes == 4:
            return 46 * n * nxh, 3 * spec + 16.25 * spec_s
        return 30 * n * nxh, 3 * spec + 13 * spec_s
    return None, None


KERNEL_NAMES = {"mv_yinv": "k_ypass<inv,2> (matvec y-inverse)", "mv_x": "k_mv_x (fused matvec x-pass)",
                "mv_yfwd": "k_ypass<fwd,EpiMatvec> (matvec y-forward + M^-1)",
                "rhs_yinv": "k_ypass<inv,4> (RHS y-inverse)", "rhs_x": "k_rhs_x (fused RHS x-pass)",
                "rhs_yfwd": "k_ypass<fwd,EpiK> (RHS y-forward)", "rk": "k_rk_update (RK4 stage update)",
                "ref_yinv": "k_ypass<inv,2> (refinement matvec y-inverse)",
                "ref_x": "k_mv_x (refinement matvec x-pass)",
                "ref_yfwd": "k_ypass<fwd,EpiMatvec> (refinement matvec y-forward)"}


def class_arith(cls, prec):
    """The arithmetic a kernel class runs in for a precision: fp32, df or fp64."""
    if prec == 0:
        return "fp64"
    if cls.startswith("ref"):
        return "df" if prec >= 2 else "fp64"
    if cls == "rk":
        return "fp64"
    if prec == 3 and cls.startswith("rhs"):
        return "df"
    return "fp32"


def class_roofline(cls, n, prec, prof, peaks, peak_kind, tuning=None):
    """HBM roofline of one kernel class from the library's per-launch CUDA-event
    timers: algorithmic bytes per launch / mean launch time, against the
    measured copy bandwidth. The FLOP rate is reported beside it."""
    cnt = prof["counts"].get(cls, 0)
    if not cnt:
        return None
    avg_ms = prof["ms"][cls] / cnt
    ar = class_arith(cls, prec)
    # the RK update reads FP32 K spectra when the right-hand side is FP32
    tbytes = 4 if (ar == "fp32" or (cls == "rk" and prec in (1, 2))) else 8
    flops, nbytes = kernel_work(cls, n, tbytes)
    if flops is None:
        return None
    peak = peaks.get("hbm_gbs", 6800.0)
    ach = nbytes / (avg_ms / 1e3) / 1e9
    tr = MEASURED_TRAFFIC.get((cls, ar, n))
    ty = {"fp32": "fp32", "df": "dfl", "fp64": "fp64"}[ar]
    if tr and tuning and (tuning.get(ty, {}).get(CLASS_TUNE.get(cls), {}) or {}).get("plan", 0) != 0:
        tr = None  # the capture is of the plan-0 kernel
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": tr["bytes"] if tr else None,
            "ncu_issue_active": tr.get("issue") if tr else None, "ncu_fma_pipe": tr.get("fma") if tr else None,
            "kernel": KERNEL_NAMES.get(cls, cls) + {"fp32": " FP32", "df": " double-float", "fp64": " FP64"}[ar],
            "algorithmic_bytes": nbytes, "avg_launch_us": avg_ms * 1e3, "launches": cnt,
            "fp64_equiv_tflops": flops / (avg_ms / 1e3) / 1e12,
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs (of {peak_kind})",
            "traffic_source": tr["source"] if tr else None}


def time_path(precision, guess, args, st, n, world, graph=0, learned=None, steps=None, warmup=None,
              profile=False, tune=None):
    """W warm-up steps, then K timed RK4 steps of one path; returns (solver,
    device fields, record). CUDA events on the launching stream bracket the
    timed call, with a synchronize (and a barrier across ranks) on both sides.
    profile: the host-driven loop (graph = 0) runs the timed steps with the
    library's per-launch event timers on."""
    import torch

    from paper_2306_09731_gb300.sgn import Solver
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    tune = (not args.no_tune) if tune is None else tune
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s = Solver(n, n, L_DEFAULT, L_DEFAULT, restart=20, tol=1e-10, precision=precision, guess=guess, graph=graph)
    tuning = s.autotune(10) if tune else None
    if learned is not None:
        net, in_scale, out_scale, tau_power = learned
        s.set_learned_guess(net, net.n, in_scale, out_scale, tau_power)
    stream = torch.cuda.current_stream()
    if warmup > 0:
        s.rk4_step(*f, DT, warmup)
    torch.cuda.synchronize()
    if profile and not graph:
        s.set_profiling(True)
    st0 = s.stats()
    l0 = s.profile()["launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rk4_step(*f, DT, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    st1 = s.stats()
    if profile and not graph:
        s.set_profiling(False)
    value, t_max = throughput(steps, ms / 1000.0, world)
    solves = st1["solves"] - st0["solves"]
    rec = {"value": value, "ms_per_step": t_max * 1e3 / steps, "steps": steps, "warmup": warmup,
           "precision": precision, "guess": guess, "graph": graph,
           "gmres": {"inner_matvecs_per_step": (st1["matvecs"] - st0["matvecs"]) / steps,
                     "solves": solves,
                     "iters_per_stage": (st1["matvecs"] - st0["matvecs"]) / max(solves, 1),
                     "refinements_per_stage": (st1["refinements"] - st0["refinements"]) / max(solves, 1),
                     "max_iters": st1["max_iters"]},
           "launches": prof["launches"] - l0,
           "prof": prof if (profile and not graph) else None,
           "tuning": tuning}
    return s, f, rec


# ---------------------------------------------------------------- the CPU oracle

def _oracle_env():
    """One BLAS/OpenMP thread per process: the oracle as it stands is serial
    numpy (pocketfft), and the all-cores timing runs one process per core."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "NUMEXPR_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_steps(n, warmup, steps):
    """Runs in a spawned process: `warmup` untimed, then `steps` timed whole
    oracle RK4 steps of the Gaussian hump on an n x n grid of the benchmark's
    box, continuing one trajectory. Returns (seconds per timed step, GMRES
    iterations of each timed stage)."""
    from oracle import sgn_oracle as O
    from paper_2306_09731_gb300 import inputs as I
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    G = O.Grid(n, n, L_DEFAULT, L_DEFAULT)
    s = (st.h, st.vx, st.vy, st.sigma)
    for _ in range(warmup):
        s = O.rk4_step(G, *s, DT, 1)
    times, log = [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        s = O.rk4_step(G, *s, DT, 1, log=log)
        times.append(time.perf_counter() - t0)
    return times, [i["iters"] for st4 in log for i in st4]


def _oracle_matvec_seconds(n, reps=2):
    """Runs in a spawned process: the best of `reps` timings of one oracle
    matvec M^-1 L sigma (the unit of GMRES work) on the n x n workload."""
    import numpy as np

    from oracle import sgn_oracle as O
    from paper_2306_09731_gb300 import inputs as I
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    G = O.Grid(n, n, L_DEFAULT, L_DEFAULT)
    x = np.cos(G.x)[None, :] * np.sin(G.y)[:, None]
    best = float("inf")
    for _ in range(reps + 1):
        t0 = time.perf_counter()
        O.precond_solve(G, O.elliptic_apply(G, st.h, x))
        best = min(best, time.perf_counter() - t0)
    return best


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_timing(n_target, n_sample, warmup, steps, all_cores=True):
    """Times the oracle as it stands on the host: `steps` whole RK4 steps of
    the workload on an n_sample^2 grid (after `warmup`), in a spawned
    one-thread process, scaled to n_target^2 by the measured ratio of one
    oracle matvec at the two sizes; with all_cores, also one step in each of
    `cores` concurrent one-thread processes (throughput of the whole host)."""
    import multiprocessing as mp
    _oracle_env()
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        times, iters = pool.apply(_oracle_steps, (n_sample, warmup, steps))
        if n_target != n_sample:
            t_big = pool.apply(_oracle_matvec_seconds, (n_target,))
            t_small = pool.apply(_oracle_matvec_seconds, (n_sample,))
            scale = t_big / t_small
        else:
            scale = 1.0
    step_s = sum(times) / len(times)
    out = {"sample_steps": steps, "sample_warmup": warmup, "sample_grid": [n_sample, n_sample],
           "sample_s_per_step": step_s, "scale_to_target": scale,
           "scale_nlogn": (n_target ** 2 * math.log2(n_target ** 2)) / (n_sample ** 2 * math.log2(n_sample ** 2)),
           "target_s_per_step": step_s * scale, "value": 1.0 / (step_s * scale),
           "iters_per_stage": sum(iters) / max(len(iters), 1), "timed_s": sum(times)}
    if all_cores:
        cores = host_cores()
        with ctx.Pool(cores) as pool:
            # one untimed step in every worker first (imports, FFT plans)
            pool.starmap(_oracle_steps, [(n_sample, 0, 1)] * cores)
            t0 = time.perf_counter()
            res = pool.starmap(_oracle_steps, [(n_sample, 0, 1)] * cores)
            wall = time.perf_counter() - t0
        per = [r[0][0] for r in res]
        out["all_cores"] = {"cores": cores, "value": cores / (wall * scale), "unit": UNIT,
                            "wall_s": wall, "mean_s_per_step_per_core": sum(per) / len(per),
                            "sample": f"one {n_sample}x{n_sample} oracle RK4 step in each of {cores} concurrent "
                                      f"one-thread processes, scaled x{scale:.2f} to {n_target}x{n_target}"}
    return out


def cpu_sample_text(t, n_target):
    return (f"{t['sample_steps']} whole oracle RK4 steps (FP64 numpy, GMRES(20) to 1e-10, "
            f"{t['iters_per_stage']:.2f} iterations per stage) of the same workload on a "
            f"{t['sample_grid'][0]}x{t['sample_grid'][1]} grid, after {t['sample_warmup']} untimed; "
            f"scaled x{t['scale_to_target']:.2f} to {n_target}x{n_target} by the measured time of one oracle "
            f"matvec at both sizes (N log N would give x{t['scale_nlogn']:.2f})")


# ---------------------------------------------------------------- extras (--full)

def time_crossing(st, precision, guess, graph, learned, steps, warmup, tune=True):
    """Wall time of `steps` graph-mode RK4 steps (after `warmup`) of one GMRES
    start on a crossing-soliton state; CUDA events on the launching stream."""
    import torch

    from paper_2306_09731_gb300.sgn import Solver
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, restart=20, tol=1e-10, precision=precision, guess=guess, graph=graph)
    if tune:
        s.autotune(5)
    if learned is not None:
        net, in_scale, out_scale, tau_power = learned
        s.set_learned_guess(net, net.n, in_scale, out_scale, tau_power)
    s.rk4_step(*f, DT, warmup)
    torch.cuda.synchronize()
    st0 = s.stats()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rk4_step(*f, DT, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    st1 = s.stats()
    solves = st1["solves"] - st0["solves"]
    s.close()
    return {"value": steps / (ms / 1000.0), "ms_per_step": ms / steps,
            "iters_per_stage": (st1["matvecs"] - st0["matvecs"]) / max(solves, 1),
            "refinements_per_stage": (st1["refinements"] - st0["refinements"]) / max(solves, 1),
            "max_iters": st1["max_iters"]}


def transverse_stability(tend=10.0, dt=2e-3, marks=5):
    """The line solitary wave of amplitude a in {0.2, 0.5, 1.0} on 1024 x 256
    over [-60, 60) x [-15, 15) with h += 1e-2 exp(-x^2) cos(2 pi y/Ly + phi),
    to t = tend with dt, in FP64 (the paper's method), precision 1 and 3, graph
    mode, extrapolated start: the L-infinity deviation from the fitted line
    soliton (Section 4.1) and the relative mass and energy drift (Section 2.3,
    from the state after the first step) at `marks` times, and the final
    difference between the precisions."""
    import numpy as np
    import torch

    from paper_2306_09731_gb300 import inputs as I
    from paper_2306_09731_gb300.sgn import Solver
    nsteps = int(round(tend / dt)) - 1
    per = nsteps // marks
    out = {}
    for a in (0.2, 0.5, 1.0):
        st = I.perturbed_soliton(1024, 256, 120.0, 30.0, a=a, eps=1e-2, seed=0)
        fin = {}
        for prec in (0, 1, 3):
            s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, precision=prec, guess=2, graph=1)
            f = [torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
                 for x in (st.h, st.vx, st.vy, st.sigma)]
            # the input sigma is 0: drifts are measured from the first step on,
            # once sigma solves its equation for the state (the energy contains it)
            s.rk4_step(*f, dt, 1)
            inv0 = s.invariants(*f)
            rows = []
            t0 = time.perf_counter()
            for k in range(1, marks + 1):
                s.rk4_step(*f, dt, per)
                inv = s.invariants(*f)
                d = s.diagnostics(f[0], f[1], f[2])
                rows.append({"t": round((1 + k * per) * dt, 6), "dev_h": d["dev_h"], "x_s": d["x_s"],
                             "mass_drift": (inv[0] - inv0[0]) / abs(inv0[0]),
                             "energy_drift": (inv[3] - inv0[3]) / abs(inv0[3])})
            torch.cuda.synchronize()
            fin[prec] = [x.cpu().numpy() for x in f[:3]]
            out.setdefault(f"a={a}", {})[{0: "fp64", 1: "mixed", 3: "precision3"}[prec]] = {
                "marks": rows, "wall_s": time.perf_counter() - t0}
            s.close()
        for p, key in ((1, "mixed_vs_fp64_rel_l2"), (3, "precision3_vs_fp64_rel_l2")):
            out[f"a={a}"][key] = {nm: float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))
                                  for nm, x, y in zip(("h", "vx", "vy"), fin[p], fin[0])}
    return {"grid": [1024, 256], "box": [[-60.0, 60.0], [-15.0, 15.0]], "eps": 1e-2, "dt": dt, "t_end": tend,
            "runs": out}


def unet_cost(reps=20):
    """Device time of one learned-start network use (batch 1): the tensor-core
    inference against the CUDA-core forward, for the library's default
    network and the four-level one, on 128^2 and 256^2 coarse grids."""
    import torch

    from paper_2306_09731_gb300.unet import SPEC_ARCH, UNet
    out = {"unit": "ms per use", "reps": reps}
    for label, arch in (("default_60705", None), ("four_level_471873", SPEC_ARCH)):
        for coarse in (128, 256):
            net = UNet(coarse, max_batch=1, bf16=True, seed=0, arch=arch)
            x = torch.randn(1, 4, coarse, coarse, device="cuda")
            y = torch.empty(1, 1, coarse, coarse, device="cuda")
            rec = {"params": net.num_params()}
            # the solver's graph mode replays the inference inside its step graph
            gs = torch.cuda.Stream()
            gs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(gs):
                net.infer(x, y)
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=gs):
                    net.infer(x, y)
            torch.cuda.current_stream().wait_stream(gs)
            for kind, fn in (("tensor_cores", lambda: net.infer(x, y)), ("tensor_cores_graph", graph.replay),
                             ("cuda_cores", lambda: net.forward(x))):
                for _ in range(3):
                    fn()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                a.record()
                for _ in range(reps):
                    fn()
                b.record()
                torch.cuda.synchronize()
                rec[kind] = a.elapsed_time(b) / reps
            net.check()
            net.close()
            out[f"{label}_n{coarse}"] = rec
    return out


def run_extras(args, st, n, detail):
    """The other arms, the learned start, the 64-member ensemble and the
    4096^2 crossing solitons; results go to the detail record only."""
    import torch

    from paper_2306_09731_gb300 import inputs as I
    arms = {}
    plan = (("mixed_df_graph", 2, 2, 1), ("mixed_df3_poly_graph", 3, 3, 1), ("fp64_poly", 0, 3, 0),
            ("mixed_df_paper_start", 2, 0, 0))
    for name, prec, guess, graph in plan:
        s, f, rec = time_path(prec, guess, args, st, n, 1, graph)
        s.close()
        rec.pop("prof", None)
        arms[name] = rec
        del f
    detail["arms"] = arms
    nets = {}
    from paper_2306_09731_gb300 import learned as Lm
    from paper_2306_09731_gb300.unet import SPEC_ARCH
    detail["unet_cost"] = unet_cost()
    lr = {}
    for name, prec, guess, graph, tau_power, coarse, warm in (
            ("mixed_df_paper_start_learned", 2, 0, 0, 1, n // 16, 1),
            ("mixed_df_learned_graph", 2, 2, 1, 2, n // 16, 1),
            ("mixed_df_poly_learned_graph", 2, 3, 1, 2, n // 16, 4)):
        t0 = time.perf_counter()
        states = Lm.gaussian_states(n, L_DEFAULT, [0.35, 0.45, 0.55, 0.65], seed=1)
        samples = Lm.generate(states, coarse, steps=8, dt=DT, precision=prec, guess=guess, tau_power=tau_power,
                              warmup=warm)
        t1 = time.perf_counter()
        net, in_scale, out_scale, losses = Lm.train(samples, iters=400, batch=8, lr=2e-3, seed=2, log_every=100,
                                                    arch=SPEC_ARCH)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        nets[name] = (net, in_scale, out_scale, tau_power)
        s, f, rec = time_path(prec, guess, args, st, n, 1, graph, nets[name])
        s.close()
        rec.pop("prof", None)
        rec["training"] = {"coarse_n": coarse, "samples": int(samples.shape[0]), "data_s": t1 - t0,
                           "train_s": t2 - t1, "losses": losses, "params": net.num_params()}
        lr[name] = rec
    detail["learned_start"] = lr
    from paper_2306_09731_gb300.ensemble import GRIDS, Ensemble, perturbed_members
    members = perturbed_members(64, seed=11)
    ens = {"members": len(members), "grids": [list(g[:2]) for g in GRIDS], "dt": 2e-3, "steps": args.steps,
           "unit": "member-steps/s"}
    for guess in (2, 3):
        E = Ensemble(members, tune=not args.no_tune, precision=2, guess=guess, graph=1)
        E.step(2e-3, max(4, args.warmup))
        torch.cuda.synchronize()
        b0 = time.perf_counter()
        E.step(2e-3, args.steps)
        b1 = time.perf_counter()
        E.step_one_by_one(2e-3, args.steps)
        b2 = time.perf_counter()
        ens[f"guess{guess}"] = {"batch": len(members) * args.steps / (b1 - b0),
                                "one_by_one": len(members) * args.steps / (b2 - b1)}
        E.close()
    # how busy the batched graphs keep the GPU: grid-point-steps/s of each
    # grid size stepped alone (one member) and batched (its members only),
    # of the whole batch, and of the 2048^2 headline (whose kernels fill the
    # GPU); the per-point work of the smaller grids is lower by their shorter
    # transforms (log2 N of 16-19 against 22)
    occ = {"unit": "grid-point-steps/s", "grids": {}}
    for g in GRIDS:
        sub = [m for m in members if (m.Nx, m.Ny) == tuple(g[:2])]
        pts = g[0] * g[1]
        for label, group in (("alone", sub[:1]), ("batched", sub)):
            E = Ensemble(group, tune=not args.no_tune, precision=2, guess=3, graph=1)
            E.step(2e-3, 4)
            torch.cuda.synchronize()
            b0 = time.perf_counter()
            E.step(2e-3, args.steps)
            wall = time.perf_counter() - b0
            its = [s.stats() for s in E.solvers]
            E.close()
            occ["grids"].setdefault(f"{g[0]}x{g[1]}", {})[label] = {
                "members": len(group), "value": len(group) * pts * args.steps / wall,
                "iters_per_stage": sum(x["matvecs"] for x in its) / max(sum(x["solves"] for x in its), 1)}
    E = Ensemble(members, tune=not args.no_tune, precision=2, guess=3, graph=1)
    E.step(2e-3, 4)
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    E.step(2e-3, args.steps)
    wall = time.perf_counter() - b0
    E.close()
    occ["all_batched"] = sum(m.Nx * m.Ny for m in members) * args.steps / wall
    if "headline" in detail:
        occ["headline_2048"] = detail["headline"]["value"] * n * n
    ens["occupancy"] = occ
    detail["ensemble"] = ens
    torch.cuda.empty_cache()
    if n == N_DEFAULT:
        ksteps = max(3, args.steps // 4)
        cross = {"workload": "crossing_solitons_4096x4096", "a": 0.6, "precision": 2, "graph": True,
                 "steps": ksteps, "theta": {}}
        for theta in (15.0, 30.0):
            cst = I.crossing_solitons(4096, 200.0, 0.6, theta)
            res = {}
            for name, guess, lname in (("paper_start", 0, None),
                                       ("paper_start_learned", 0, "mixed_df_paper_start_learned"),
                                       ("extrapolated", 2, None), ("extrapolated_learned", 2, "mixed_df_learned_graph"),
                                       ("polynomial", 3, None),
                                       ("polynomial_learned", 3, "mixed_df_poly_learned_graph")):
                res[name] = time_crossing(cst, 2, guess, 1, nets.get(lname), ksteps, 4 if guess == 3 else 2,
                                          not args.no_tune)
            cross["theta"][f"{theta:g}"] = res
            del cst
        detail["crossing_4096"] = cross


def compact_line(head_rec, fp64, roof, share, e2e, clk, args, world, n):
    """The one JSON object the bench prints last: the headline, the paper's
    method beside it, the roofline of the dominant kernel, the end-to-end
    figure and the clocks (a few KB; every table goes to the detail file)."""
    prec, guess, graph = head_rec["precision"], head_rec["guess"], head_rec["graph"]
    out = {
        "metric": METRIC, "value": head_rec["value"], "unit": UNIT, "n_gpus": world, "steps": head_rec["steps"],
        "warmup": head_rec["warmup"], "ms_per_step": head_rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+df64+f64", "data": "synthetic",
        "config": dict(config(n, HEADLINE_PATH), parallelism=f"replicas{world}" if world > 1 else "single",
                       precision_id=prec, guess=guess, graph=graph, tuned=not args.no_tune),
        "gmres": {k: head_rec["gmres"][k] for k in ("iters_per_stage", "refinements_per_stage", "max_iters")},
        "gpu_launches": head_rec["launches"],
        "fp64_plain": fp64,
        "speedup_vs_fp64": (head_rec["value"] / fp64["value"]) if fp64 else None,
        "roofline": ({k: roof.get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "traffic", "kernel",
                                                "avg_launch_us", "algorithmic_bytes", "time_share",
                                                "fp64_equiv_tflops", "ncu_issue_active", "ncu_fma_pipe",
                                                "peak_source", "traffic_source")} if roof else None),
        "e2e": e2e,
        "clocks": clk,
    }
    if share:
        top = sorted(share.items(), key=lambda kv: -kv[1])[:5]
        out["time_share_top"] = {k: round(v, 4) for k, v in top}
    return out


# ---------------------------------------------------------------- our arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2306_09731_gb300 import inputs as I
    from paper_2306_09731_gb300.sgn import sgn_rk4_step_host

    torch.cuda.set_device(local_rank)
    n = args.n
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    peaks, peak_kind = measured_peaks()
    detail = {"metric": METRIC, "n": n}

    # the headline, timed on its own with the clocks sampled around it
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.4)
    prec, guess, graph = HEADLINE
    head, hf, head_rec = time_path(prec, guess, args, st, n, world, graph)
    clk = clocks.stop()
    head_fields = [x.cpu().numpy() for x in hf[:3]]
    detail["headline"] = {k: v for k, v in head_rec.items() if k != "prof"}

    # end to end through the C ABI with host buffers: every step copies the
    # state in from pinned host memory and the result back (in the call)
    e2e_steps = args.steps if args.e2e_steps is None else args.e2e_steps
    nbytes = 4 * n * n * 8
    e2e = None
    if e2e_steps > 0:
        pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory().numpy()
        hh = [pin(st.h), pin(st.vx), pin(st.vy), pin(st.sigma)]
        sgn_rk4_step_host(head.handle, *hh, DT, 1)  # warm
        for _ in range(max(0, args.warmup - 1)):
            sgn_rk4_step_host(head.handle, *hh, DT, 1)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            sgn_rk4_step_host(head.handle, *hh, DT, 1)
        w1 = time.perf_counter()
        e2e_value, _ = throughput(e2e_steps, w1 - w0, world)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "steps": e2e_steps, "api": "sgn_rk4_step_host, pinned host buffers, one step per call"}
    head.close()
    del hf

    # the paper's method: FP64 throughout, GMRES from the last sigma, host loop
    fp64 = None
    if not args.no_fp64:
        s, f, rec = time_path(0, 0, args, st, n, world, 0)
        s.close()
        ff = [x.cpu().numpy() for x in f[:3]]
        del f
        fp64 = {"value": rec["value"], "ms_per_step": rec["ms_per_step"],
                "iters_per_stage": rec["gmres"]["iters_per_stage"], "path": "precision 0, guess 0, host loop"}
        fp64["headline_vs_fp64_rel_l2"] = {
            nm: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
            for nm, a, b in zip(("h", "vx", "vy"), head_fields, ff)}
        fp64["after_steps"] = args.warmup + args.steps
        detail["fp64_plain"] = {k: v for k, v in rec.items() if k != "prof"}

    # the headline's kernels in the host-driven loop with per-launch CUDA-event
    # timers: the roofline of the dominant kernel and the time shares
    roof, share = None, None
    if not args.no_prof:
        s, f, rec = time_path(prec, guess, args, st, n, world, 0, profile=True)
        s.close()
        del f
        prof = rec["prof"]
        rl = {c: class_roofline(c, n, prec, prof, peaks, peak_kind, rec.get("tuning")) for c in SINGLE_KERNEL_CLASSES}
        rl = {c: r for c, r in rl.items() if r}
        total = sum(prof["ms"].values())
        share = {k: v / total for k, v in prof["ms"].items() if v > 0}
        gm = sum(prof["ms"].get(k, 0.0) for k in ("mv_yinv", "mv_x", "mv_yfwd", "krylov", "ref_yinv", "ref_x",
                                                  "ref_yfwd"))
        if rl:
            dom = max(rl, key=lambda c: prof["ms"][c])
            roof = dict(rl[dom])
            roof["time_share"] = share[dom]
        detail["profiled_host_loop"] = {"value": rec["value"], "ms_per_step": rec["ms_per_step"],
                                        "gmres": rec["gmres"], "time_share": share,
                                        "gmres_share": gm / total if total else None,
                                        "kernel_ms_per_step": total / rec["steps"], "rooflines": rl}

    if args.full and world == 1:
        run_extras(args, st, n, detail)
    if args.transverse and world == 1:
        detail["transverse"] = transverse_stability()

    out = compact_line(head_rec, fp64, roof, share, e2e, clk, args, world, n)
    return out, detail


# ---------------------------------------------------------------- reference arm

def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle as it stands (the paper ships no
    code), rank 0 only. Each step is one whole oracle RK4 step of the workload
    at --sample-n, scaled to the --n grid by the measured matvec cost ratio."""
    if rank != 0:
        return None
    n, ns = args.n, min(args.sample_n, args.n)
    t = oracle_timing(n, ns, args.warmup, args.steps, all_cores=True)
    cb = {"value": t["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": cpu_sample_text(t, n)}
    return {"metric": METRIC, "value": t["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup,
            # the time each timed step actually took (a sample step); the value
            # is the scaled steps/s of the full-size workload
            "ms_per_step": t["sample_s_per_step"] * 1e3,
            "ms_per_step_scaled": t["target_s_per_step"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": dict(config(n, "fp64 (the paper's method, CPU oracle)"), parallelism="single",
                           sample_grid=[ns, ns]),
            "cpu_baseline": cb, "all_cores": t.get("all_cores"),
            "e2e": {"value": t["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def write_detail(path, detail):
    try:
        d = os.path.dirname(path)
        if d:
            os.makedirs(d, exist_ok=True)
        with open(path, "w") as f:
            json.dump(detail, f, indent=1, default=str)
        return path
    except OSError as e:
        print(f"bench: could not write {path}: {e}", file=sys.stderr)
        return None


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, detail = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a bounded sample: 2 whole oracle steps at 512^2 on one core, then one
        # step on every core at once
        t = oracle_timing(args.n, min(args.sample_n, args.n), 1, 2, all_cores=True)
        out["cpu_baseline"] = {"value": t["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": cpu_sample_text(t, args.n),
                               "all_cores": {k: t["all_cores"][k] for k in ("cores", "value", "unit")}}
        detail["cpu_baseline"] = t
    if rank == 0:
        out["detail"] = write_detail(args.detail, dict(detail, line=out))
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
