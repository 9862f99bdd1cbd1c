"""Ensembles of independent problems stepped together (sgn_rk4_step_batch).

Each member has its own handle, grid and CUDA stream; with graph mode the
library enqueues every member's steps before waiting for any, so members on
their own streams run concurrently. This module only builds members and
marshals arguments.
"""
import numpy as np

from . import inputs as I
from .sgn import Solver, sgn_rk4_step_batch

# uneven grids of the perturbed-soliton ensemble: (Nx, Ny, Lx, Ly)
GRIDS = [(256, 256, 60.0, 60.0), (512, 256, 120.0, 60.0), (1024, 512, 120.0, 60.0)]


def perturbed_members(count, seed=0, grids=GRIDS):
    """count perturbed line solitons, a ~ U[0.1, 1], eps ~ U[1e-3, 5e-2], grids
    cycling through `grids`; returns the initial states."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        Nx, Ny, Lx, Ly = grids[i % len(grids)]
        a = float(rng.uniform(0.1, 1.0))
        eps = float(rng.uniform(1e-3, 5e-2))
        out.append(I.perturbed_soliton(Nx, Ny, Lx, Ly, a=a, eps=eps, seed=int(rng.integers(1 << 30))))
    return out


class Ensemble:
    """Handles, streams and device fields of a list of initial states."""

    def __init__(self, states, tune=False, **opts):
        """tune: run sgn_autotune on each member's handle (launch shapes for
        its grid; members of the ensemble's small grids gain the most)."""
        import torch
        self._torch = torch
        self.states = states
        self.streams = [torch.cuda.Stream() for _ in states]
        self.solvers = []
        self.fields = []
        self.tuning = []
        for st, s in zip(states, self.streams):
            sol = Solver(st.Nx, st.Ny, st.Lx, st.Ly, **opts)
            sol.set_stream(s)
            if tune:
                self.tuning.append(sol.autotune(3))
            self.solvers.append(sol)
            self.fields.append([torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
                                for a in (st.h, st.vx, st.vy, st.sigma)])
        torch.cuda.synchronize()

    def step(self, dt, nsteps):
        """Every member nsteps steps together; returns the member statuses."""
        return sgn_rk4_step_batch([s.handle for s in self.solvers], self.fields, dt, nsteps)

    def step_one_by_one(self, dt, nsteps):
        for s, f in zip(self.solvers, self.fields):
            s.rk4_step(*f, dt, nsteps)

    def close(self):
        for s in self.solvers:
            s.close()
        self.solvers = []
