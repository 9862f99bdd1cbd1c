"""The premise of the polynomial GMRES start (guess = 3), on the oracle.

With a fixed dt, the sigma that RK4 stage s solves for is a smooth function of
the step's start time, so its values at the last steps predict the next step's
by the polynomial through them, with the error of that polynomial: O(dt^3) for
the quadratic through 3 steps (backward-difference weights 3, -3, 1) and
O(dt^4) for the cubic through 4 (4, -6, 4, -1). Halving dt must then cut the
prediction error by about 8 and 16, against 4 for the linear extrapolation
inside a step. A wrong weight (or a wrong step order) drops the order and
fails the ratio. The last test shows, with FP32 emulated by rounding, why the
FP32 right-hand side adds its linear part in FP64: rounded whole, its noise
would dominate the cubic start's error near rest.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2306_09731_gb300 import inputs as I

WEIGHTS = {2: (2.0, -1.0), 3: (3.0, -3.0, 1.0), 4: (4.0, -6.0, 4.0, -1.0)}


def stage_sigmas(G, h, vx, vy, dt, nsteps):
    """sigma of each RK4 stage of each step (solved to 1e-14)."""
    sig = np.zeros_like(h)
    out = []
    for _ in range(nsteps):
        U = (h, vx, vy)
        Ks, sigs = [], []
        for s in range(4):
            if s == 0:
                Y = U
            else:
                c = dt if s == 3 else 0.5 * dt
                Y = tuple(u + c * k for u, k in zip(U, Ks[-1]))
            ht, vxt, vyt, sig, _ = O.rhs(G, *Y, sig, tol=1e-14)
            Ks.append((ht, vxt, vyt))
            sigs.append(sig)
        out.append(sigs)
        h, vx, vy = (u + dt / 6.0 * (a + 2.0 * b + 2.0 * c + d) for u, a, b, c, d in zip(U, *Ks))
    return out


def prediction_errors(dt, steps=5):
    G = O.Grid(32, 32, 8.0, 8.0)
    st = I.random_state(32, 32, 8.0, 8.0, seed=5, kmax=3)
    phi = I.random_smooth(32, 32, 8.0, 8.0, seed=6, kmax=3)
    sig = stage_sigmas(G, st.h, O.dx(G, phi), O.dy(G, phi), dt, steps)
    errs = {}
    for order, w in WEIGHTS.items():
        e = 0.0
        for s in range(4):
            pred = sum(wk * sig[steps - 2 - k][s] for k, wk in enumerate(w))
            true = sig[steps - 1][s]
            e = max(e, float(np.linalg.norm(pred - true) / np.linalg.norm(true)))
        errs[order] = e
    return errs


@pytest.fixture(scope="module")
def errors():
    return prediction_errors(8e-3), prediction_errors(4e-3)


@pytest.mark.parametrize("order,ratio", [(2, 3.0), (3, 6.0), (4, 11.0)])
def test_extrapolation_error_order(errors, order, ratio):
    coarse, fine = errors
    assert coarse[order] / fine[order] > ratio, (coarse, fine)


def test_cubic_beats_quadratic_beats_linear(errors):
    for e in errors:
        assert e[4] < e[3] < e[2]


# ----------------------------------------------------------------------------
# Why the FP32 right-hand side leaves its linear part to the FP64 update.
# Rounding the whole right-hand side (and its input state) to FP32 puts noise
# into every stage state that changes from step to step without pattern; the
# cubic weights amplify it, and near rest (v = 0 at t = 0), where sigma is
# small, it dominates the start's error. Rounding only the nonlinear part
# keeps the start as accurate as with the exact right-hand side.

def _f32(a):
    return a.astype(np.float32).astype(np.float64)


def _rhs_linear(G, h, vx, vy, s, g=1.0):
    """The part of the right-hand side linear in the state: h_t from
    q = v - grad sigma, v_t = -grad g (h - 1)."""
    qx, qy = vx - O.dx(G, s), vy - O.dy(G, s)
    return -(O.dx(G, qx) + O.dy(G, qy)), -g * O.dx(G, h - 1.0), -g * O.dy(G, h - 1.0)


def _rhs_full(G, h, vx, vy, s, g=1.0):
    sx, sy = O.dx(G, s), O.dy(G, s)
    ux, uy = vx - sx / h, vy - sy / h
    ht = -(O.dx(G, h * ux) + O.dy(G, h * uy))
    F = 0.5 * (vx ** 2 + vy ** 2) - (sx ** 2 + sy ** 2) / (2.0 * h ** 2) + g * (h - 1.0) \
        - 4.5 * s ** 2 / h ** 4
    return ht, -O.dx(G, F), -O.dy(G, F)


def _cubic_start_error(mode, dt=4e-3, steps=7):
    G = O.Grid(32, 32, 8.0, 8.0)
    st = I.gaussian_hump(32, 8.0, 0.5)
    h, vx, vy = st.h, st.vx, st.vy
    sig = np.zeros_like(h)
    hist = []
    for _ in range(steps):
        U = (h, vx, vy)
        Ks, sigs = [], []
        for s in range(4):
            Y = U if s == 0 else tuple(u + (dt if s == 3 else 0.5 * dt) * k for u, k in zip(U, Ks[-1]))
            sig, _, _, _ = O.gmres(G, Y[0], O.divergence_rhs(G, Y[1], Y[2]), sig, tol=1e-14)
            sigs.append(sig)
            if mode == "exact":
                K = _rhs_full(G, *Y, sig)
            else:
                r = (1.0 + _f32(Y[0] - 1.0), _f32(Y[1]), _f32(Y[2]), _f32(sig))
                if mode == "fp32":
                    K = tuple(_f32(k) for k in _rhs_full(G, *r))
                else:  # split: FP32 nonlinear part, exact linear part
                    K = tuple(a + _f32(b - c) for a, b, c in
                              zip(_rhs_linear(G, *Y, sig), _rhs_full(G, *r), _rhs_linear(G, *r)))
            Ks.append(K)
        hist.append(sigs)
        h, vx, vy = (u + dt / 6.0 * (a + 2.0 * b + 2.0 * c + d) for u, a, b, c, d in zip(U, *Ks))
    w = WEIGHTS[4]
    return max(float(np.linalg.norm(sum(wk * hist[steps - 2 - k][s] for k, wk in enumerate(w))
                                    - hist[steps - 1][s]) / np.linalg.norm(hist[steps - 1][s]))
               for s in range(4))


def test_linear_part_in_fp64_keeps_the_cubic_start():
    exact, fp32, split = (_cubic_start_error(m) for m in ("exact", "fp32", "split"))
    assert split < 1.5 * exact
    assert fp32 > 10.0 * split
