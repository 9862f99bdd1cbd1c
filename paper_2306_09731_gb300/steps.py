"""Run RK4 steps of the Gaussian-hump workload in one configuration.

    python -m paper_2306_09731_gb300.steps --n 2048 --precision 2 --guess 3 \
        --graph 0 --warmup 4 --steps 2

h = 1 + 0.5 exp(-(x^2+y^2)), v = 0 on [-50, 50)^2 (the benchmark's state),
dt = 1e-3, GMRES restart 20, tol 1e-10. Runs `warmup` steps in one call and
then `steps` more in a second call, and prints the kernels launched and the
GMRES statistics of the second call. Meant as a small fixed command to run
under a profiler (the host-driven loop, graph 0, launches every kernel on its
own; graph mode replays each step as one CUDA graph).
"""
from __future__ import annotations

import argparse
import json


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=int, default=2048, help="grid points per side")
    ap.add_argument("--precision", type=int, default=2)
    ap.add_argument("--guess", type=int, default=3)
    ap.add_argument("--graph", type=int, default=0)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--tune", action="store_true", help="sgn_autotune the handle first")
    args = ap.parse_args(argv)

    import torch

    from . import inputs as I
    from .sgn import Solver

    n, L = args.n, 100.0
    st = I.gaussian_hump(n, L, 0.5)
    s = Solver(n, n, L, L, precision=args.precision, guess=args.guess, graph=args.graph)
    if args.tune:
        s.autotune(5)
    f = [torch.tensor(a, dtype=torch.float64, device="cuda").contiguous() for a in (st.h, st.vx, st.vy, st.sigma)]
    if args.warmup > 0:
        s.rk4_step(*f, 1e-3, args.warmup)
    torch.cuda.synchronize()
    l0 = s.profile()["launches"]
    s0 = s.stats()
    if args.steps > 0:
        s.rk4_step(*f, 1e-3, args.steps)
    torch.cuda.synchronize()
    s1 = s.stats()
    launches = s.profile()["launches"] - l0
    s.close()
    print(json.dumps({"launches": launches,
                      "matvecs": s1["matvecs"] - s0["matvecs"], "solves": s1["solves"] - s0["solves"],
                      "refinements": s1["refinements"] - s0["refinements"], "last_relres": s1["last_relres"]}))


if __name__ == "__main__":
    main()
