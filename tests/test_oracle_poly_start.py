"""The premise of the polynomial GMRES start (guess = 3), on the oracle.

With a fixed dt, the sigma that RK4 stage s solves for is a smooth function of
the step's start time, so its values at the last steps predict the next step's
by the polynomial through them, with the error of that polynomial: O(dt^3) for
the quadratic through 3 steps (backward-difference weights 3, -3, 1) and
O(dt^4) for the cubic through 4 (4, -6, 4, -1). Halving dt must then cut the
prediction error by about 8 and 16, against 4 for the linear extrapolation
inside a step. A wrong weight (or a wrong step order) drops the order and
fails the ratio.
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
