"""Run the learned start's network on the tensor cores in one configuration.

    python -m paper_2306_09731_gb300.infer --n 256 --batch 8 --reps 3

Creates the four-level network of 471,873 parameters (or the library's default
one with --default), runs sgn_unet_infer `reps` times on a seeded random input
[batch][4][n][n] and prints the device time of the last call and the kernels
one call launches. Meant as a small fixed command to run under a profiler.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=256, help="coarse grid side")
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--default", action="store_true", help="the library's default network")
    args = ap.parse_args(argv)

    import torch

    from .unet import SPEC_ARCH, UNet

    net = UNet(args.n, max_batch=args.batch, bf16=True, seed=0, arch=None if args.default else SPEC_ARCH)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(args.batch, 4, args.n, args.n, device="cuda", generator=g)
    y = torch.empty(args.batch, 1, args.n, args.n, device="cuda")
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(max(args.reps - 1, 0)):
        net.infer(x, y)
    a.record()
    net.infer(x, y)
    b.record()
    torch.cuda.synchronize()
    net.check()
    levels, widths = net.arch()
    out = {"n": args.n, "batch": args.batch, "levels": levels, "widths": list(widths), "params": net.num_params(),
           "ms": a.elapsed_time(b), "launches_per_call": 4 * levels - 1}
    net.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
