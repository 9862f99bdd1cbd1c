"""Host-side parts of bench.py that need no GPU.

The reference arm (the oracle, timed on the host cores) prints one JSON line
with the keys the bench's contract names, and its steps and ms_per_step are
the work it actually timed. Rank 0 alone runs it. The line the bench prints
last is compact and carries the contract's keys. The algorithmic byte model
of the roofline is checked against its definition: spectra of the stated
types, per launch.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CONTRACT_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config", "e2e")


def test_reference_arm_json_line():
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "64", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    wall = time.perf_counter() - t0
    assert out.returncode == 0, out.stderr
    line = out.stdout.strip().splitlines()[-1]
    d = json.loads(line)
    for key in CONTRACT_KEYS + ("impl", "cpu_baseline"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    # the claimed timed region (steps x ms_per_step) fits in the command's wall time
    assert d["steps"] * d["ms_per_step"] / 1e3 < wall
    # no sample scaling when the sample is the workload itself
    assert abs(d["ms_per_step_scaled"] - d["ms_per_step"]) < 1e-9
    assert d["config"]["precision"].startswith("fp64")
    assert d["all_cores"]["cores"] >= 1 and d["all_cores"]["value"] > 0


def test_reference_arm_other_ranks_do_nothing():
    import bench
    args = argparse.Namespace(n=64, sample_n=64, steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2) is None


def test_compact_line_keys_and_size():
    """The last stdout line: the contract's keys, the paper's method beside the
    headline, and a few KB at most (the driver keeps only the output's tail)."""
    import bench
    gm = {"iters_per_stage": 1.25, "refinements_per_stage": 1.0, "max_iters": 7, "inner_matvecs_per_step": 5.0,
          "solves": 80}
    head = {"value": 180.0, "ms_per_step": 5.55, "steps": 20, "warmup": 5, "precision": 2, "guess": 3, "graph": 1,
            "gmres": gm, "launches": 4000}
    fp64 = {"value": 13.8, "ms_per_step": 72.4, "iters_per_stage": 6.1, "path": "precision 0, guess 0, host loop",
            "headline_vs_fp64_rel_l2": {"h": 1e-12, "vx": 2e-9, "vy": 4e-9}, "after_steps": 25}
    roof = bench.class_roofline("ref_x", 2048, 2, {"ms": {"ref_x": 2.9}, "counts": {"ref_x": 10}},
                                {"hbm_gbs": 6777.6}, "measured")
    roof["time_share"] = 0.24
    e2e = {"value": 120.0, "unit": "steps/s", "h2d_bytes_per_step": 4 * 2048 * 2048 * 8,
           "d2h_bytes_per_step": 4 * 2048 * 2048 * 8, "steps": 20, "api": "sgn_rk4_step_host"}
    clk = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 30}
    args = bench.parse(["--steps", "20", "--warmup", "5"])
    out = bench.compact_line(head, fp64, roof, {"ref_x": 0.24, "rk": 0.1}, e2e, clk, args, 1, 2048)
    for key in CONTRACT_KEYS + ("roofline", "clocks", "gpu_launches", "fp64_plain"):
        assert key in out, key
    assert out["config"]["workload"] == "gaussian_hump_2048x2048"
    assert abs(out["speedup_vs_fp64"] - 180.0 / 13.8) < 1e-12
    r = out["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert len(json.dumps(out)) < 4096


def test_summarize_clocks():
    import bench
    lines = ["0, 2070, 2070, 500.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    c = bench.summarize_clocks(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["reasons"] == ["sw_power_cap"]


def test_kernel_byte_model():
    import bench
    n = 2048
    nxh = n // 2 + 1
    spec32, spec64 = n * nxh * 8, n * nxh * 16
    # matvec y-inverse: sigma_hat read, sigma and i ky sigma written (FP32 pass)
    assert bench.kernel_work("mv_yinv", n, 4)[1] == 3 * spec32
    # refinement x-pass in double-float: 4 spectra and 2 coefficient fields at 8 bytes
    assert bench.kernel_work("ref_x", n, 8)[1] == 4 * spec64 + 2 * n * n * 8
    # FP32 RK update: K (3 FP32 spectra), 13 FP64 state spectra, and on
    # average 3.25 more for the right-hand side's linear part
    assert bench.kernel_work("rk", n, 4)[1] == 3 * spec32 + 16.25 * spec64
    assert bench.kernel_work("rk", n, 8)[1] == 3 * spec64 + 13 * spec64
    # arithmetic of each class per precision
    assert bench.class_arith("ref_x", 2) == "df" and bench.class_arith("mv_x", 2) == "fp32"
    assert bench.class_arith("rhs_x", 3) == "df" and bench.class_arith("rk", 2) == "fp64"
    assert bench.class_arith("mv_x", 0) == "fp64"


def test_measured_traffic_matches_its_profile_summary():
    """Every DRAM figure the roofline reports as `traffic` names a summary
    under profiles/, and that summary's table carries the same read and write
    megabytes for the kernel (so a kernel change that leaves an old figure in
    the bench, or a summary that no longer backs it, fails here)."""
    import re

    import bench
    for (cls, arith, n), tr in bench.MEASURED_TRAFFIC.items():
        path = os.path.join(ROOT, tr["source"])
        assert os.path.isfile(path), tr["source"]
        text = open(path).read()
        pairs = {(float(a), float(b)) for a, b in re.findall(r"\|\s*([\d.]+)\s*/\s*([\d.]+)\s*\|", text)}
        assert any(abs((a + b) * 1e6 - tr["bytes"]) < 0.06e6 for a, b in pairs), (cls, arith, n, tr["bytes"])
        assert 0.0 < tr["issue"] <= 1.0 and 0.0 < tr["fma"] <= 1.0
