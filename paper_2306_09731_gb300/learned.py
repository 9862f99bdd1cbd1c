"""Training of the learned GMRES start on snapshots the solver generates.

Section 3 starts GMRES from the last computed sigma. The learned start adds a
network's correction to that start at RK4 stages 2 and 4, or at every stage
over the polynomial start of guess 3 (include/sgn.h, sgn_set_learned_guess).
This module orchestrates its training; every computation runs in the
library's kernels: the solver records coarse samples
(sgn_record_learned) and the U-Net kernels (include/sgn_unet.h) run the
forward pass, the backward pass and Adam.

Sample channels (coarse n x n): h - 1, vx, vy, sigma_start and the target
(sigma_solved - sigma_start) / tau, tau = (dt/2)^tau_power. Inputs are scaled
to unit RMS and the target by its RMS; the scales go to the solver with the
network.
"""
import numpy as np

from . import inputs as I
from .sgn import Solver
from .unet import UNet


def gaussian_states(N, L, amplitudes, seed=0):
    """Gaussian humps h = 1 + a exp(-r^2), v = 0, centred at a seeded random grid point."""
    rng = np.random.default_rng(seed)
    out = []
    for a in amplitudes:
        st = I.gaussian_hump(N, L, float(a))
        sy, sx = (int(v) for v in rng.integers(-N // 8, N // 8, size=2))
        st.h = np.roll(st.h, (sy, sx), axis=(0, 1))
        out.append(st)
    return out


def generate(states, coarse, steps, dt, precision=2, guess=0, tau_power=1, warmup=1):
    """Runs each state for warmup + steps RK4 steps, recording the steps;
    returns the samples [S][5][coarse][coarse] (CUDA float32). With guess 3
    the solver records only once its polynomial start is cubic, 4 steps into
    a trajectory whose history every other library call restarts: the
    warm-up and the recorded steps then run as one call (give warmup >= 4)."""
    import torch
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    parts = []
    for st in states:
        s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, precision=precision, guess=guess)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        if guess == 3:
            buf = s.record_learned(coarse, 4 * (steps + warmup), tau_power)
            s.rk4_step(*f, dt, warmup + steps)
        else:
            if warmup:
                s.rk4_step(*f, dt, warmup)
            buf = s.record_learned(coarse, 4 * steps, tau_power)
            s.rk4_step(*f, dt, steps)
        count = s.stop_recording()
        parts.append(buf[:count].clone())
        s.close()
    return torch.cat(parts)


def scales(samples):
    """(in_scale[4], out_scale): reciprocal RMS of each input channel and the target's RMS."""
    rms = samples.double().pow(2).mean(dim=(0, 2, 3)).sqrt().cpu().numpy()
    in_scale = [float(1.0 / r) if r > 0 else 1.0 for r in rms[:4]]
    out_scale = float(rms[4]) if rms[4] > 0 else 1.0
    return in_scale, out_scale


def train(samples, iters=600, batch=8, lr=2e-3, seed=0, log_every=0, arch=None):
    """Adam on the mean squared error of the scaled target; returns
    (net, in_scale, out_scale, losses) with one loss per log_every iterations.
    arch = (levels, widths) of the network (None: the library's default)."""
    import torch
    coarse = samples.shape[-1]
    in_scale, out_scale = scales(samples)
    sc = torch.tensor(in_scale, dtype=torch.float32, device="cuda")[None, :, None, None]
    X = (samples[:, :4] * sc).contiguous()
    T = (samples[:, 4:5] / out_scale).contiguous()
    S = samples.shape[0]
    batch = min(batch, S)
    net = UNet(coarse, max_batch=batch, bf16=True, seed=seed, arch=arch)
    rng = np.random.default_rng(seed)
    losses = []
    for t in range(1, iters + 1):
        idx = torch.tensor(rng.choice(S, batch, replace=False), device="cuda")
        net.forward(X[idx].contiguous())
        loss = net.backward(T[idx].contiguous())
        if log_every and (t == 1 or t % log_every == 0):
            losses.append(loss)
        net.adam_step(lr, t)
    return net, in_scale, out_scale, losses


def attach(solver, net, in_scale, out_scale, tau_power):
    solver.set_learned_guess(net, net.n, in_scale, out_scale, tau_power)
