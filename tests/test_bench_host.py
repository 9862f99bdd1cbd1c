"""Host-side parts of bench.py that need no GPU.

The reference arm (the oracle, timed on one host core) prints one JSON line
with the keys the bench's contract names. Rank 0 alone runs it. The
algorithmic byte model of the roofline is checked against its definition:
spectra of the stated types, per launch.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "64", "--steps", "2",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_other_ranks_do_nothing():
    import argparse

    import bench
    args = argparse.Namespace(n=64, steps=1, warmup=0)
    assert bench.run_reference(args, 1, 2) is None


def test_kernel_byte_model():
    import bench
    n = 2048
    nxh = n // 2 + 1
    spec32, spec64 = n * nxh * 8, n * nxh * 16
    # matvec y-inverse: sigma_hat read, sigma and i ky sigma written (FP32 pass)
    assert bench.kernel_work("mv_yinv", n, 4)[1] == 3 * spec32
    # FP32 RK update: K (3 FP32 spectra), 13 FP64 state spectra, and on
    # average 3.25 more for the right-hand side's linear part
    assert bench.kernel_work("rk", n, 4)[1] == 3 * spec32 + 16.25 * spec64
    assert bench.kernel_work("rk", n, 8)[1] == 3 * spec64 + 13 * spec64
