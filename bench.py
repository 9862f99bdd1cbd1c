#!/usr/bin/env python
"""Benchmark: 2D SGN RK4 steps/s on the 2048^2 Gaussian-hump workload.

Workload: h = 1 + 0.5 exp(-(x^2+y^2)), v = 0 on [-50,50)^2, 2048 x 2048 points,
dt = 1e-3, GMRES restart 20 and tolerance 1e-10 (FP64 path). One step is one
classic RK4 step (4 RHS evaluations, each with its GMRES solve), the whole hot
path. Inputs are resident in HBM when the timed region starts; the state and
the Krylov basis (about 1.3 GB) are far larger than L2, so no flush is needed.

Prints ONE JSON line on rank 0. Under torchrun every rank steps its own
replica (weak scaling, no collective on the data path); value = total steps of
all ranks / max time over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (each
step is a bounded sample: one RK4 stage, scaled x4).
"""
from __future__ import annotations

import argparse
import json
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_DEFAULT, help="grid points per side (default 2048)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-graph", action="store_true", help="skip the graph-mode arms")
    ap.add_argument("--no-df", action="store_true", help="skip the double-float refinement arms")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-start arms (and their training)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 64-member ensemble measurement")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the built-in launch shapes (no sgn_autotune before the warm-up)")
    ap.add_argument("--transverse", action="store_true",
                    help="also run the transverse-stability workload to t = 10 (1024x256, FP64 and precision 1)")
    ap.add_argument("--no-crossing", action="store_true",
                    help="skip the 4096^2 crossing-soliton measurement (GMRES starts compared)")
    ap.add_argument("--arms", default=None, help="comma list: run only these arms (mixed, mixed_graph, mixed_df, "
                                                 "mixed_df_graph, fp64, mixed_paper_start, mixed_df3_graph, "
                                                 "mixed_df_poly, mixed_df_poly_graph, mixed_df3_poly_graph, "
                                                 "fp64_poly)")
    ap.add_argument("--path", choices=["both", "mixed", "fp64"], default="both",
                    help="headline is the mixed path when it runs; both also times plain FP64")
    return ap.parse_args()


def config(n, fp32=False):
    return {"workload": f"gaussian_hump_{n}x{n}", "grid": [n, n], "box": [-L_DEFAULT / 2, L_DEFAULT / 2],
            "h0": f"1+{ALPHA}*exp(-(x^2+y^2))", "v0": "0", "dt": DT, "gmres_restart": 20, "gmres_tol": 1e-10,
            "precision": ("fp32 transforms/pointwise/inner GMRES, fp64 state, dots, Givens and refinement "
                          "residual" if fp32 else "fp64"),
            "l2": "inputs larger than L2 (state + Krylov basis, 0.9-1.3 GB), no flush"}


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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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


# FP64 rate of a GB300: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz max clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# Double-float passes (precision 2) are bound by FP32 issue: 152 SMs x 128 FP32
# lanes x 2.07 GHz instructions per second, divided by the FP32 instructions
# one FP64-equivalent flop of a radix-8 FFT butterfly costs in this
# double-float arithmetic: (52 adds x 8 + 4 products x 7 + 7 complex twiddle
# products x 38) / (52 + 4 + 7 x 6) = 7.2.
DF_INSTR_PER_FLOP = (52 * 8 + 4 * 7 + 7 * 38) / (52 + 4 + 7 * 6)
DF_PEAK_TFLOPS = 152 * 128 * 2.07e9 / DF_INSTR_PER_FLOP / 1e12

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# is now, with the summary that holds the command; set to None when the kernel
# changes.
MEASURED_TRAFFIC = {
    ("ref_x", "df", 2048): {"bytes": 134.603264e6 + 22.911744e6, "source": "profiles/k_mv_x_df_gaussian2048.md"},
    ("mv_x", "fp32", 2048): {"bytes": 67.196928e6 + 0.668928e6, "source": "profiles/k_mv_x_fp32_gaussian2048.md"},
    ("mv_yinv", "fp32", 2048): {"bytes": 16.893696e6 + 0.13824e6, "source": "profiles/k_ypass_fp32_gaussian2048.md"},
    ("mv_yfwd", "fp32", 2048): {"bytes": 33.669888e6 + 0.076288e6, "source": "profiles/k_ypass_fp32_gaussian2048.md"},
    ("rhs_yinv", "fp32", 2048): {"bytes": 102.639616e6 + 31.659264e6,
                                 "source": "profiles/k_ypass_fp32_gaussian2048.md"},
    ("rhs_yfwd", "fp32", 2048): {"bytes": 50.482688e6 + 3.486976e6,
                                 "source": "profiles/k_ypass_fp32_gaussian2048.md"},
    ("mv_x", "fp64", 2048): {"bytes": 134.8608e6 + 29.78304e6, "source": "profiles/k_mv_x_fp64_gaussian2048.md"},
}

# kernel classes that are one kernel each (candidates for the roofline line)
SINGLE_KERNEL_CLASSES = ("mv_x", "mv_yinv", "mv_yfwd", "rhs_x", "rhs_yinv", "rhs_yfwd", "rk", "ref_yinv", "ref_x",
                         "ref_yfwd")


def kernel_work(cls, n, tbytes):
    """Algorithmic (flops, DRAM bytes) of one launch of a kernel class at n x n.

    tbytes: bytes per real of the pass (8 FP64, 4 FP32); the RK4 state, sigma
    and b stay FP64 (8) in both modes. FFT flops: 5 m log2 m per complex
    transform of length m, 2.5 m log2 m per real one.
    """
    import math
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


def class_roofline(cls, n, prec, prof, peaks):
    """Live roofline of one kernel class from the library's event timers."""
    cnt = prof["counts"].get(cls, 0)
    if not cnt:
        return None
    avg_ms = prof["ms"][cls] / cnt
    is32 = prec >= 1 and not cls.startswith("ref")
    isdf = prec == 2 and cls.startswith("ref")
    flops, nbytes = kernel_work(cls, n, 4 if is32 else 8)
    if flops is None:
        return None
    if isdf:
        ach = flops / (avg_ms / 1e3) / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": ach / DF_PEAK_TFLOPS,
               "peak_source": "derived double-float rate: 152 SMs x 128 FP32 lanes x 2.07 GHz / "
                              f"{DF_INSTR_PER_FLOP:.1f} FP32 instructions per FP64-equivalent FFT flop"}
    elif is32:
        ach = nbytes / (avg_ms / 1e3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        out = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
               "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    else:
        ach = flops / (avg_ms / 1e3) / 1e12
        out = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "frac": ach / FP64_PEAK_TFLOPS,
               "peak_source": "derived FP64 rate: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz"}
    out.update({"kernel": KERNEL_NAMES.get(cls, cls) + (" FP32" if is32 else (" double-float" if isdf else " FP64")),
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": nbytes,
                "avg_launch_ms": avg_ms, "launches": cnt})
    tr = MEASURED_TRAFFIC.get((cls, "fp32" if is32 else ("df" if isdf else "fp64"), n))
    out["traffic"] = tr["bytes"] if tr else None
    out["traffic_source"] = tr["source"] if tr else None
    return out


def time_path(precision, guess, args, st, n, world, graph=0, learned=None):
    """W warm-up steps, then K timed RK4 steps of one path; returns its record.

    The host-driven loop (graph = 0) runs the timed steps with the per-launch
    event timers on; graph mode (graph = 1) cannot time launches inside its
    conditional nodes and runs without them."""
    import torch

    from paper_2306_09731_gb300.sgn import Solver
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s = Solver(n, n, L_DEFAULT, L_DEFAULT, restart=20, tol=1e-10, precision=precision, guess=guess, graph=graph)
    tuning = None if args.no_tune else s.autotune(5)
    if learned is not None:
        net, in_scale, out_scale, tau_power = learned
        s.set_learned_guess(net, net.n, in_scale, out_scale, tau_power)
    stream = torch.cuda.current_stream()
    if args.warmup > 0:
        s.rk4_step(*f, DT, args.warmup)
    torch.cuda.synchronize()
    if not graph:
        s.set_profiling(True)
    st0 = s.stats()
    l0 = s.profile()["launches"]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rk4_step(*f, DT, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    st1 = s.stats()
    if not graph:
        s.set_profiling(False)
    value, t_max = throughput(args.steps, ms / 1000.0, world)
    solves = st1["solves"] - st0["solves"]
    rec = {"value": value, "ms_per_step": t_max * 1e3 / args.steps,
           "gmres": {"inner_matvecs_per_step": (st1["matvecs"] - st0["matvecs"]) / args.steps,
                     "solves": solves,
                     "iters_per_stage": (st1["matvecs"] - st0["matvecs"]) / max(solves, 1),
                     "fp64_refinements_per_stage": (st1["refinements"] - st0["refinements"]) / max(solves, 1)},
           "launches": prof["launches"] - l0,
           "prof": None if graph else prof,
           "tuning": tuning}
    return s, f, rec


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
            "fp64_refinements_per_stage": (st1["refinements"] - st0["refinements"]) / max(solves, 1),
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


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2306_09731_gb300 import inputs as I
    from paper_2306_09731_gb300.sgn import sgn_rk4_step_host

    torch.cuda.set_device(local_rank)
    n = args.n
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    peaks, _ = measured_peaks()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.4)
    paths = {}
    fields = {}
    # mixed: FP32 bulk + FP64 refinement, GMRES started by linear extrapolation in
    # time, host-driven loop with per-launch timers (the per-kernel rooflines);
    # mixed_df: the same with the refinement matvec and the coefficient pass in
    # double-float arithmetic (precision 2); *_graph: the same kernels with each
    # RK4 step replayed as a CUDA graph; fp64: the paper's method (FP64, start
    # from the last sigma); mixed_paper_start: precision 1 with the paper's
    # start, for attribution; *_poly*: each stage started from the polynomial
    # in time through the same stage's sigma of the last 3-4 steps (guess 3)
    plan = (("mixed", 1, 2, 0), ("mixed_graph", 1, 2, 1), ("mixed_df", 2, 2, 0), ("mixed_df_graph", 2, 2, 1),
            ("fp64", 0, 0, 0), ("mixed_paper_start", 1, 0, 0), ("mixed_df3_graph", 3, 2, 1),
            ("mixed_df_poly", 2, 3, 0), ("mixed_df_poly_graph", 2, 3, 1), ("mixed_df3_poly_graph", 3, 3, 1),
            ("fp64_poly", 0, 3, 0))
    solvers = {}
    devfields = {}
    for name, prec, guess, graph in plan:
        if args.path == "mixed" and not name.startswith("mixed"):
            continue
        if args.path == "fp64" and not name.startswith("fp64"):
            continue
        if args.no_graph and graph:
            continue
        if args.no_df and prec == 2:
            continue
        if args.arms and name not in args.arms.split(","):
            continue
        s, f, rec = time_path(prec, guess, args, st, n, world, graph)
        rec["precision"] = prec
        fields[name] = [x.cpu().numpy() for x in f[:3]]
        devfields[name] = f
        solvers[name] = s
        paths[name] = rec
    # learned start: networks trained here on solver snapshots of four
    # other Gaussian humps (amplitudes 0.35-0.65, shifted centres), then run on
    # the benchmark state: over the paper's start (tau = dt/2, coarse n/8) and
    # over the extrapolated start (tau = (dt/2)^2, coarse n/16)
    learned_info = {}
    nets = {}
    if not args.no_learned and args.path != "fp64" and (not args.arms or any("learned" in a for a in
                                                                              args.arms.split(","))):
        from paper_2306_09731_gb300 import learned as Lm
        for name, prec, guess, graph, tau_power, coarse in (
                ("mixed_df_paper_start", 2, 0, 0, 0, 0), ("mixed_df_paper_start_learned", 2, 0, 0, 1, n // 8),
                ("mixed_df_learned_graph", 2, 2, 1, 2, n // 16)):
            if args.arms and name not in args.arms.split(","):
                continue
            learned = None
            if coarse:
                t0 = time.perf_counter()
                states = Lm.gaussian_states(n, L_DEFAULT, [0.35, 0.45, 0.55, 0.65], seed=1)
                samples = Lm.generate(states, coarse, steps=8, dt=DT, precision=prec, guess=guess,
                                      tau_power=tau_power)
                t1 = time.perf_counter()
                net, in_scale, out_scale, losses = Lm.train(samples, iters=400, batch=8, lr=2e-3, seed=2,
                                                            log_every=100)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                learned = (net, in_scale, out_scale, tau_power)
                nets[name] = learned
                learned_info[name] = {"coarse_n": coarse, "samples": int(samples.shape[0]),
                                      "data_s": t1 - t0, "train_s": t2 - t1, "losses": losses,
                                      "params": net.num_params()}
            s, f, rec = time_path(prec, guess, args, st, n, world, graph, learned)
            rec["precision"] = prec
            fields[name] = [x.cpu().numpy() for x in f[:3]]
            devfields[name] = f
            solvers[name] = s
            paths[name] = rec
    # headline: the fastest arm of the headline path (all of them meet the same
    # FP64 tolerance test in every solve); its per-kernel figures come from the
    # host-driven arm of the same precision
    if args.path == "fp64":
        head_name = "fp64"
    else:
        cands = [k for k in ("mixed", "mixed_graph", "mixed_df", "mixed_df_graph", "mixed_df_learned_graph",
                             "mixed_df_poly", "mixed_df_poly_graph") if k in paths]
        head_name = max(cands, key=lambda k: paths[k]["value"])
    prof_name = {"mixed_graph": "mixed", "mixed_df_graph": "mixed_df", "mixed_df_learned_graph": "mixed_df",
                 "mixed_df_poly_graph": "mixed_df_poly"}.get(head_name, head_name)
    head_solver, head_rec = solvers[head_name], paths[head_name]
    head_prec = head_rec["precision"]
    for name, s in solvers.items():
        if name != head_name:
            s.close()
    clk = clocks.stop()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, args.steps // 4)
    nbytes = 4 * n * n * 8
    e2e = None
    if e2e_steps > 0:
        pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory().numpy()
        hh = [pin(st.h), pin(st.vx), pin(st.vy), pin(st.sigma)]
        sgn_rk4_step_host(head_solver.handle, *hh, DT, 1)  # warm
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            sgn_rk4_step_host(head_solver.handle, *hh, DT, 1)
        w1 = time.perf_counter()
        e2e_value, _ = throughput(e2e_steps, w1 - w0, world)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
               "api": "sgn_rk4_step_host (pinned host buffers, one step per call)"}
    # ensembles: 64 perturbed line solitons, a ~ U[0.1, 1], eps ~ U[1e-3, 5e-2], on
    # 256^2, 512x256 and 1024x512 grids, dt = 2e-3, each member with its own handle and
    # stream: sgn_rk4_step_batch against the members stepped one by one (wall time of
    # K steps of all members after W warm-up steps; host timers around calls that
    # synchronise)
    ensemble = None
    if not args.no_ensemble and world == 1 and args.path != "fp64" and not args.arms:
        from paper_2306_09731_gb300.ensemble import GRIDS, Ensemble, perturbed_members
        members = perturbed_members(64, seed=11)
        ens = {}
        for tuned in ((False, True) if not args.no_tune else (False,)):
            E = Ensemble(members, tune=tuned, precision=2, guess=2, graph=1)
            E.step(2e-3, max(1, args.warmup))
            torch.cuda.synchronize()
            b0 = time.perf_counter()
            E.step(2e-3, args.steps)
            b1 = time.perf_counter()
            E.step_one_by_one(2e-3, args.steps)
            b2 = time.perf_counter()
            ens[tuned] = (b1 - b0, b2 - b1, E.tuning[:3] if tuned else None)
            E.close()
        tb, to, tuning = ens[max(ens)]
        ensemble = {"members": len(members), "grids": [list(g[:2]) for g in GRIDS], "dt": 2e-3,
                    "steps": args.steps, "unit": "member-steps/s",
                    "batch": len(members) * args.steps / tb,
                    "one_by_one": len(members) * args.steps / to,
                    "speedup": to / tb, "tuned": max(ens)}
        if True in ens and False in ens:
            ensemble["batch_builtin_shapes"] = len(members) * args.steps / ens[False][0]
            ensemble["tuning_first_members"] = tuning
        # the same batch with the polynomial start (4 warm-up steps of history)
        E = Ensemble(members, tune=max(ens), precision=2, guess=3, graph=1)
        E.step(2e-3, max(4, args.warmup))
        torch.cuda.synchronize()
        b0 = time.perf_counter()
        E.step(2e-3, args.steps)
        ensemble["batch_polynomial"] = len(members) * args.steps / (time.perf_counter() - b0)
        E.close()
    # the paper's monitoring quantities on the final state: wall time of
    # one sgn_diagnostics call (three max sweeps, one 3-field FFT, one readback)
    hf = devfields[head_name]
    head_solver.diagnostics(hf[0], hf[1], hf[2])
    torch.cuda.synchronize()
    d0 = time.perf_counter()
    for _ in range(5):
        diag = head_solver.diagnostics(hf[0], hf[1], hf[2])
    diag_ms = (time.perf_counter() - d0) / 5 * 1e3
    head_solver.close()

    # crossing line solitons at 4096^2 (the learned start's workload): two a = 0.6
    # solitons rotated by +-theta, precision 2, graph mode, every solve to the
    # FP64 tolerance 1e-10; the paper's start (last sigma), the extrapolated
    # start, and each with the network trained above on the 2048^2 Gaussian
    # snapshots (coarse grids 256 and 128)
    crossing = None
    if not args.no_crossing and world == 1 and args.path != "fp64" and not args.arms and n == N_DEFAULT:
        del devfields, hf
        torch.cuda.empty_cache()
        ksteps, kwarm = max(3, args.steps // 4), 2
        crossing = {"workload": "crossing_solitons_4096x4096", "grid": [4096, 4096], "box": [-100.0, 100.0],
                    "a": 0.6, "dt": DT, "precision": 2, "graph": True, "steps": ksteps,
                    "warmup": kwarm, "warmup_polynomial": max(kwarm, 4),
                    "unit": UNIT, "tol": 1e-10, "theta": {}}
        for theta in (15.0, 30.0):
            cst = I.crossing_solitons(4096, 200.0, 0.6, theta)
            arms = {}
            # the polynomial start needs 4 steps of history before the cubic:
            # its arm warms up for 4 steps
            for name, guess, lname in (("paper_start", 0, None),
                                       ("paper_start_learned", 0, "mixed_df_paper_start_learned"),
                                       ("extrapolated", 2, None),
                                       ("extrapolated_learned", 2, "mixed_df_learned_graph"),
                                       ("polynomial", 3, None)):
                if lname is not None and lname not in nets:
                    continue
                arms[name] = time_crossing(cst, 2, guess, 1, nets.get(lname), ksteps,
                                           max(kwarm, 4) if guess == 3 else kwarm, not args.no_tune)
            crossing["theta"][f"{theta:g}"] = arms
            del cst
        for ln, (net, *_rest) in nets.items():
            crossing.setdefault("networks", {})[ln] = {"coarse_n": net.n}

    fp32 = head_prec >= 1
    # a run restricted to graph arms (--arms) has no per-launch timers
    prof = paths[prof_name]["prof"] if prof_name in paths else {"ms": {}, "counts": {}, "launches": 0}
    rooflines = {c: class_roofline(c, n, head_prec, prof, peaks) for c in SINGLE_KERNEL_CLASSES}
    doms = [c for c in rooflines if rooflines[c]]
    dom = max(doms, key=lambda c: prof["ms"][c]) if doms else None
    total_prof = sum(prof["ms"].values())
    gmres_ms = sum(prof["ms"].get(k, 0.0) for k in ("mv_yinv", "mv_x", "mv_yfwd", "krylov", "ref_yinv", "ref_x",
                                                    "ref_yfwd"))
    out = {
        "metric": METRIC, "value": head_rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head_rec["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if fp32 else "f64", "data": "synthetic",
        "config": dict(config(n, fp32), parallelism=f"replicas{world}" if world > 1 else "single"),
        "path": ({0: "plain FP64",
                  1: "mixed: FP32 bulk + FP64 refinement to the FP64 tolerance",
                  2: "mixed: FP32 bulk + double-float refinement matvec and coefficients to the FP64 tolerance"}
                 [head_prec])
                + (", GMRES start: each stage's sigma extrapolated by the cubic in time through the same stage "
                   "of the last 4 steps" if "_poly" in head_name else ", GMRES start extrapolated in time")
                + (", each RK4 step one CUDA graph with device-side GMRES control"
                   if head_name.endswith("_graph") else ", host-driven GMRES loop"),
        "arms": {k: dict({"value": v["value"], "ms_per_step": v["ms_per_step"], "precision": v["precision"],
                          "graph": k.endswith("_graph"), "iters_per_stage": v["gmres"]["iters_per_stage"],
                          "tuned_threads": ({ty: {ps: r["threads"] for ps, r in d.items()}
                                             for ty, d in v["tuning"].items()} if v.get("tuning") else None)},
                         **({"avg_launch_ms": {c: v["prof"]["ms"][c] / v["prof"]["counts"][c]
                                               for c in v["prof"]["ms"] if v["prof"]["counts"][c]}}
                            if v["prof"] else {}))
                 for k, v in paths.items()},
        "gmres": head_rec["gmres"],
        # launch shapes sgn_autotune picked for the headline handle, with the
        # timed launch (us) of each pass in the built-in and the picked shape
        "tuning": head_rec.get("tuning"),
        "time_share": {k: v / total_prof for k, v in prof["ms"].items() if v > 0},
        "gmres_share": gmres_ms / total_prof if total_prof else None,
        # kernel time summed from the event timers of the host-driven run: the
        # rest of its ms_per_step is launch gaps and the per-Arnoldi-step host
        # synchronisation
        "kernel_ms_per_step": total_prof / args.steps,
        "gpu_launches": head_rec["launches"],
        # time_share and the rooflines come from the host-driven run of the same
        # kernels (graph mode has no per-launch timers)
        "roofline_source": f"{prof_name} (host-driven loop, CUDA events per launch)",
        "roofline": rooflines[dom] if dom else None,
        "roofline_by_kernel": {c: {"frac": r["frac"], "bound": r["bound"], "achieved": r["achieved"],
                                   "unit": r["unit"], "avg_launch_ms": r["avg_launch_ms"]}
                               for c, r in rooflines.items() if r},
        "e2e": e2e,
        "clocks": clk,
        "diagnostics": {"ms_per_call": diag_ms, "h_max": diag["h_max"], "c_fit": diag["c_fit"],
                        "tail": diag["tail"]},
        "ensemble": ensemble,
        "crossing_4096": crossing,
        "transverse": transverse_stability() if (args.transverse and world == 1) else None,
    }
    if "fp64_poly" in paths:
        fp = paths["fp64_poly"]
        out["fp64_poly_start"] = {"value": fp["value"], "unit": UNIT, "ms_per_step": fp["ms_per_step"],
                                  "gmres": fp["gmres"]}
    if "fp64" in paths and head_name != "fp64":
        f64 = paths["fp64"]
        out["fp64_plain"] = {"value": f64["value"], "unit": UNIT, "ms_per_step": f64["ms_per_step"],
                             "gmres": f64["gmres"]}
        out["speedup_vs_fp64"] = head_rec["value"] / f64["value"]
        errs = {}
        for i, nm in enumerate(("h", "vx", "vy")):
            a, b = fields[head_name][i], fields["fp64"][i]
            errs[nm] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        out["headline_vs_fp64_rel_l2"] = errs
        out["headline_vs_fp64_after_steps"] = args.warmup + args.steps
    for base in ("mixed", "mixed_df", "mixed_df_poly"):
        if base + "_graph" in paths and base in paths:
            mg, mh = paths[base + "_graph"], paths[base]
            out.setdefault("graph_vs_host_loop", {})[base] = {
                "graph": mg["value"], "host_loop": mh["value"], "unit": UNIT, "ratio": mg["value"] / mh["value"],
                "fields_bitwise_equal": all(bool(np.array_equal(a, b))
                                            for a, b in zip(fields[base + "_graph"], fields[base]))}
    if learned_info:
        lr = {"training": learned_info}
        for base, arm in (("mixed_df_paper_start", "mixed_df_paper_start_learned"),
                          ("mixed_df_graph", "mixed_df_learned_graph")):
            if base in paths and arm in paths:
                b, a = paths[base], paths[arm]
                lr[arm] = {"value": a["value"], "base": base, "base_value": b["value"],
                           "speedup": a["value"] / b["value"],
                           "inner_matvecs_per_step": a["gmres"]["inner_matvecs_per_step"],
                           "base_inner_matvecs_per_step": b["gmres"]["inner_matvecs_per_step"],
                           "refinements_per_stage": a["gmres"]["fp64_refinements_per_stage"],
                           "base_refinements_per_stage": b["gmres"]["fp64_refinements_per_stage"]}
        out["learned_start"] = lr
    if "mixed_paper_start" in paths:
        mp = paths["mixed_paper_start"]
        out["mixed_paper_start"] = {"value": mp["value"], "unit": UNIT, "ms_per_step": mp["ms_per_step"],
                                    "gmres": mp["gmres"]}
    return out


def oracle_stage_sample(n):
    """Times one RK4 stage of the oracle (stage 2 of the first step) at n x n."""
    import numpy as np

    from oracle import sgn_oracle as O
    from paper_2306_09731_gb300 import inputs as I
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    G = O.Grid(n, n, L_DEFAULT, L_DEFAULT)
    k1h, k1x, k1y, sig, _ = O.rhs(G, st.h, st.vx, st.vy, st.sigma)
    t0 = time.perf_counter()
    _, _, _, _, info = O.rhs(G, st.h + 0.5 * DT * k1h, st.vx + 0.5 * DT * k1x, st.vy + 0.5 * DT * k1y, sig)
    t = time.perf_counter() - t0
    return t, info["iters"]


def run_reference(args, rank, world):
    if rank != 0:
        return None
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    n = args.n
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_stage_sample(min(n, 256))
    times = []
    its = []
    for _ in range(args.steps):
        t, it = oracle_stage_sample(n)
        times.append(t)
        its.append(it)
    step_s = 4.0 * sum(times) / len(times)
    value = 1.0 / step_s
    sample = (f"{args.steps} samples of one RK4 stage (stage 2 of step 1, {its[0]} GMRES iterations) of the "
              f"{n}x{n} workload, step time = 4 x mean stage time")
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": dict(config(n, True), parallelism="single"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if args.steps > 3 and args.n >= 2048:
            args.steps = 3  # each sample is ~20-30 s of single-core work
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_ours(args, rank, world, local_rank)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        t, it = oracle_stage_sample(args.n)
        v = 1.0 / (4.0 * t)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"one RK4 stage (stage 2 of step 1, {it} GMRES iterations, FP64) of the "
                                         f"{args.n}x{args.n} workload, x4 for a step; numpy FFT, 1 thread"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
