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
    return ap.parse_args()


def config(n):
    return {"workload": f"gaussian_hump_{n}x{n}", "grid": [n, n], "box": [-L_DEFAULT / 2, L_DEFAULT / 2],
            "h0": f"1+{ALPHA}*exp(-(x^2+y^2))", "v0": "0", "dt": DT, "gmres_restart": 20, "gmres_tol": 1e-10,
            "precision": "fp64", "l2": "inputs larger than L2 (state + Krylov basis ~1.3 GB), no flush"}


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

# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# is now, with the summary that holds the command; set to None when the kernel
# changes.
MEASURED_TRAFFIC = {
    ("mv_x", "fp64", 2048): {"bytes": 134.508544e6 + 23.561472e6,
                             "source": "profiles/k_mv_x_fp64_gaussian2048.md"},
}

# kernel classes that are one kernel each (candidates for the roofline line)
SINGLE_KERNEL_CLASSES = ("mv_x", "mv_yinv", "mv_yfwd", "rhs_x", "rhs_yinv", "rhs_yfwd")


def mv_x_flops(n):
    """Algorithmic flops of one launch of the fused matvec x-pass at n x n.

    Per row: 3 inverse and 3 forward real FFTs of length n (2.5 n log2 n each),
    plus the pointwise products (6 per point) and the a - i kx b combination
    (4 per half-spectrum entry).
    """
    import math
    rows = n
    return rows * (6 * 2.5 * n * math.log2(n) + 6 * n + 4 * (n // 2 + 1))


def mv_x_bytes(n):
    """Algorithmic DRAM bytes of one launch: read S, Sy (2 half spectra) and the
    two coefficient fields, write C, By (2 half spectra), FP64."""
    spec = n * (n // 2 + 1) * 16
    phys = n * n * 8
    return 4 * spec + 2 * phys


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2306_09731_gb300 import inputs as I
    from paper_2306_09731_gb300.sgn import Solver, sgn_rk4_step_host

    torch.cuda.set_device(local_rank)
    n = args.n
    st = I.gaussian_hump(n, L_DEFAULT, ALPHA)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    h, vx, vy, sg = dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)
    s = Solver(n, n, L_DEFAULT, L_DEFAULT, restart=20, tol=1e-10)
    stream = torch.cuda.current_stream()
    if args.warmup > 0:
        s.rk4_step(h, vx, vy, sg, DT, args.warmup)
    torch.cuda.synchronize()
    s.set_profiling(True)
    stats0 = s.stats()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.4)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.rk4_step(h, vx, vy, sg, DT, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    prof = s.profile()
    stats1 = s.stats()
    s.set_profiling(False)
    value, t_max = throughput(args.steps, ms / 1000.0, world)
    ms_max = t_max * 1000.0

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else max(3, args.steps // 4)
    nbytes = 4 * n * n * 8
    e2e = None
    if e2e_steps > 0:
        pin = lambda a: torch.tensor(a, dtype=torch.float64).pin_memory().numpy()
        hh = [pin(st.h), pin(st.vx), pin(st.vy), pin(st.sigma)]
        sgn_rk4_step_host(s.handle, *hh, DT, 1)  # warm
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        w0 = time.perf_counter()
        for _ in range(e2e_steps):
            sgn_rk4_step_host(s.handle, *hh, DT, 1)
        w1 = time.perf_counter()
        e2e_value, _ = throughput(e2e_steps, w1 - w0, world)
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
               "api": "sgn_rk4_step_host (pinned host buffers, one step per call)"}

    # roofline of the dominant kernel class
    cls = max(SINGLE_KERNEL_CLASSES, key=lambda k: prof["ms"][k])
    launches_dom = prof["counts"][cls]
    avg_ms = prof["ms"][cls] / max(launches_dom, 1)
    peaks, src = measured_peaks()
    if cls == "mv_x":
        achieved = mv_x_flops(n) / (avg_ms / 1e3) / 1e12
        roof = {"kernel": "k_mv_x (fused matvec x-pass)", "bound": "alu", "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": (MEASURED_TRAFFIC.get(("mv_x", "fp64", n)) or {}).get("bytes"),
                "traffic_source": (MEASURED_TRAFFIC.get(("mv_x", "fp64", n)) or {}).get("source"),
                "algorithmic_bytes_per_launch": mv_x_bytes(n),
                "achieved_gbs": mv_x_bytes(n) / (avg_ms / 1e3) / 1e9, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                "peak_source": "derived FP64 FMA rate (152 SMs x 2 FMA/clk x 2 x 2.07 GHz)",
                "avg_launch_ms": avg_ms, "launches": launches_dom}
    else:
        roof = {"kernel": cls, "bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": None, "traffic": None, "avg_launch_ms": avg_ms}

    matvecs = stats1["matvecs"] - stats0["matvecs"]
    solves = stats1["solves"] - stats0["solves"]
    total_prof = sum(prof["ms"].values())
    gmres_ms = sum(prof["ms"][k] for k in ("mv_yinv", "mv_x", "mv_yfwd", "krylov"))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(config(n), parallelism=f"replicas{world}" if world > 1 else "single"),
        "path": "plain FP64",
        "gmres": {"matvecs_per_step": matvecs / args.steps, "solves": solves,
                  "iters_per_stage": matvecs / max(solves, 1)},
        "time_share": {k: v / total_prof for k, v in prof["ms"].items()},
        "gmres_share": gmres_ms / total_prof if total_prof else None,
        "gpu_launches": prof["launches"],
        "roofline": roof,
        "e2e": e2e,
        "clocks": clk,
    }
    s.close()
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
            "config": dict(config(n), parallelism="single"),
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
                               "sample": f"one RK4 stage (stage 2 of step 1, {it} GMRES iterations) of the "
                                         f"{args.n}x{args.n} workload, x4 for a step; numpy FFT, 1 thread"}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
