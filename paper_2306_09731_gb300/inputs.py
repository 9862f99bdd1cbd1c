"""Seeded, synthetic initial data for the 2D SGN solver (numpy only).

This module is shared by the tests, the benchmark and the oracle's tests. It
holds the workloads' initial data and nothing of the numerical method itself
(no spectral derivative, no elliptic operator, no time stepping): every field
here is a closed-form expression evaluated on the collocation grid.

Grid convention (periodic box, full periods ``Lx``, ``Ly``):
    x_j = -Lx/2 + j*Lx/Nx,  j = 0..Nx-1;   y_l = -Ly/2 + l*Ly/Ny
Fields are numpy arrays of shape ``(Ny, Nx)`` (row-major, x fastest), float64.

Line solitary wave (Section 2.4, Eq. (sol)): with h_inf = g = 1 and amplitude a,
    c^2 = g(h_inf + a),  kappa^2 = 3a / (4 h_inf^2 (h_inf + a)),
    h_c = h_inf + a sech^2(kappa xi),  xi = x - x0 - c t,
    u_c = c + m/h_c with m = -c h_inf,
    sigma = m (h_c^2)'/6,  v = phi' = c + (m/h_c)(1 + (h_c^2)''/6).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def coords(Nx: int, Ny: int, Lx: float, Ly: float):
    """Collocation points of the periodic box [-Lx/2, Lx/2) x [-Ly/2, Ly/2)."""
    x = -0.5 * Lx + Lx * np.arange(Nx, dtype=np.float64) / Nx
    y = -0.5 * Ly + Ly * np.arange(Ny, dtype=np.float64) / Ny
    return x, y


@dataclass
class Soliton1D:
    """Closed-form line solitary wave of Eq. (sol) and its xi-derivatives."""

    a: float
    g: float = 1.0
    h_inf: float = 1.0

    @property
    def c(self) -> float:
        return math.sqrt(self.g * (self.h_inf + self.a))

    @property
    def kappa(self) -> float:
        return math.sqrt(3.0 * self.a / (4.0 * self.h_inf ** 2 * (self.h_inf + self.a)))

    def fields(self, xi: np.ndarray) -> dict:
        """h, u, v, sigma and their first xi-derivatives at travelling coordinate xi."""
        a, c, k, hi = self.a, self.c, self.kappa, self.h_inf
        m = -c * hi
        T = np.tanh(k * xi)
        S = 1.0 - T * T                      # sech^2
        S1 = -2.0 * k * S * T                # dS/dxi
        S2 = k * k * (4.0 * S - 6.0 * S * S)  # d2S/dxi2
        # third derivative: d/dxi of k^2 (4S - 6S^2) = k^2 (4 - 12 S) S'
        S3 = k * k * (4.0 - 12.0 * S) * S1
        h = hi + a * S
        h1 = a * S1
        h2 = a * S2
        h3 = a * S3
        q1 = 2.0 * h * h1                    # (h^2)'
        q2 = 2.0 * (h1 * h1 + h * h2)        # (h^2)''
        q3 = 2.0 * (3.0 * h1 * h2 + h * h3)  # (h^2)'''
        u = c + m / h
        u1 = -m * h1 / (h * h)
        sigma = m * q1 / 6.0
        sigma1 = m * q2 / 6.0
        v = c + (m / h) * (1.0 + q2 / 6.0)
        v1 = -m * h1 / (h * h) * (1.0 + q2 / 6.0) + (m / h) * (q3 / 6.0)
        return dict(h=h, u=u, v=v, sigma=sigma, h_xi=h1, u_xi=u1, v_xi=v1,
                    sigma_xi=sigma1)


@dataclass
class State:
    """Initial data on a grid. ``sigma`` is a closed form where one exists, else zeros."""

    Nx: int
    Ny: int
    Lx: float
    Ly: float
    h: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    sigma: np.ndarray
    g: float = 1.0
    meta: dict = field(default_factory=dict)


def line_soliton(Nx, Ny, Lx, Ly, a, x0=0.0, t=0.0, g=1.0) -> State:
    """y-independent line solitary wave centred at x0 + c t (Eq. (sol))."""
    sol = Soliton1D(a=a, g=g)
    x, _ = coords(Nx, Ny, Lx, Ly)
    f = sol.fields(x - x0 - sol.c * t)
    ones = np.ones((Ny, 1))
    return State(Nx, Ny, Lx, Ly, h=ones * f["h"], vx=ones * f["v"],
                 vy=np.zeros((Ny, Nx)), sigma=ones * f["sigma"], g=g,
                 meta=dict(kind="line_soliton", a=a, c=sol.c, kappa=sol.kappa,
                           x0=x0, t=t, fields=f))


def soliton_256x16(t: float = 0.0) -> State:
    """Line solitary wave a=0.5 on 256x16 points over [-40,40)x[-5,5)."""
    return line_soliton(256, 16, 80.0, 10.0, a=0.5, t=t)


def perturbed_soliton(Nx=1024, Ny=256, Lx=120.0, Ly=30.0, a=0.5, eps=1e-2,
                      seed=0) -> State:
    """Line soliton plus eps exp(-x^2) cos(2 pi y/Ly + phi), phi ~ U[0, 2pi) seeded.

    Only h is perturbed; v stays the unperturbed soliton's (curl-free) field.
    """
    st = line_soliton(Nx, Ny, Lx, Ly, a=a)
    rng = np.random.default_rng(seed)
    phi = float(rng.uniform(0.0, 2.0 * math.pi))
    x, y = coords(Nx, Ny, Lx, Ly)
    st.h = st.h + eps * np.exp(-x[None, :] ** 2) * np.cos(2 * math.pi * y[:, None] / Ly + phi)
    st.sigma = np.zeros((Ny, Nx))
    st.meta.update(kind="perturbed_soliton", eps=eps, phase=phi, seed=seed)
    return st


def gaussian_hump(N=2048, L=100.0, alpha=0.5) -> State:
    """h = 1 + alpha exp(-(x^2+y^2)), v = 0 (so sigma = 0) on [-L/2, L/2)^2."""
    x, y = coords(N, N, L, L)
    h = 1.0 + alpha * np.exp(-(x[None, :] ** 2 + y[:, None] ** 2))
    z = np.zeros((N, N))
    return State(N, N, L, L, h=h, vx=z, vy=z.copy(), sigma=z.copy(),
                 meta=dict(kind="gaussian_hump", alpha=alpha))


def gaussian_hump_flow(N=2048, L=100.0, alpha=0.5, beta=0.2) -> State:
    """The Gaussian hump h = 1 + alpha exp(-(x^2+y^2)) carrying a smooth
    potential flow v = grad(phi), phi = beta exp(-((x-1)^2 + y^2)/2) (so
    curl v = 0, the class of flows of Section 2.1), sigma = 0 as the GMRES
    start: the benchmark's depth with a right-hand side whose nonlinear
    terms are not zero."""
    x, y = coords(N, N, L, L)
    X, Y = x[None, :], y[:, None]
    h = 1.0 + alpha * np.exp(-(X ** 2 + Y ** 2))
    e = beta * np.exp(-0.5 * ((X - 1.0) ** 2 + Y ** 2))
    vx = -(X - 1.0) * e
    vy = -Y * e
    return State(N, N, L, L, h=h, vx=np.ascontiguousarray(vx), vy=np.ascontiguousarray(vy),
                 sigma=np.zeros((N, N)), meta=dict(kind="gaussian_hump_flow", alpha=alpha, beta=beta))


def deformed_soliton(Nx=1024, Ny=128, Lx=20 * math.pi, Ly=4 * math.pi, c=1.7,
                     x0=-10.0, shift=0.1) -> State:
    """Deformed line soliton of Eq. (soldef): crest at x0 + shift cos(y).

    v_x = c - (c/h)(1 + (h^2)_xx/6), v_y = 0, with (h^2)_xx taken analytically
    along x for the shifted profile.
    """
    a = c * c - 1.0
    sol = Soliton1D(a=a)
    x, y = coords(Nx, Ny, Lx, Ly)
    xi = x[None, :] - x0 - shift * np.cos(y)[:, None]
    f = sol.fields(xi)
    h = f["h"]
    # (h^2)'' along x equals the xi form because xi_x = 1
    hx = f["h_xi"]
    k = sol.kappa
    T = np.tanh(k * xi)
    S = 1.0 - T * T
    hxx = a * k * k * (4.0 * S - 6.0 * S * S)
    q2 = 2.0 * (hx * hx + h * hxx)
    vx = c - (c / h) * (1.0 + q2 / 6.0)
    return State(Nx, Ny, Lx, Ly, h=h, vx=vx, vy=np.zeros_like(h),
                 sigma=np.zeros_like(h), meta=dict(kind="deformed_soliton", c=c, x0=x0))


def random_smooth(Nx, Ny, Lx, Ly, seed=0, kmax=6, amp=0.2, mean=0.0) -> np.ndarray:
    """Seeded band-limited real field: mean + sum of cos/sin modes |m| <= kmax.

    Built from explicit separable cos/sin products, amplitudes ~ amp * N(0,1) / (1+|m|^2).
    """
    rng = np.random.default_rng(seed)
    x, y = coords(Nx, Ny, Lx, Ly)
    X = 2 * math.pi * (x + 0.5 * Lx) / Lx
    Y = 2 * math.pi * (y + 0.5 * Ly) / Ly
    mx_max = min(kmax, Nx // 2 - 1)
    my_max = min(kmax, Ny // 2 - 1)
    f = np.full((Ny, Nx), float(mean))
    for mx in range(0, mx_max + 1):
        cx, sx = np.cos(mx * X), np.sin(mx * X)
        for my in range(-my_max, my_max + 1):
            if mx == 0 and my <= 0:
                continue
            cy, sy = np.cos(my * Y), np.sin(my * Y)
            w = amp / (1.0 + mx * mx + my * my)
            p, q = rng.standard_normal(2) * w
            # cos(mx X + my Y) and sin(mx X + my Y) by angle addition
            f += p * (np.outer(cy, cx) - np.outer(sy, sx))
            f += q * (np.outer(sy, cx) + np.outer(cy, sx))
    return f


def random_state(Nx, Ny, Lx, Ly, seed=0, kmax=6, h_amp=0.15, v_amp=0.1) -> State:
    """Seeded smooth positive depth and velocity (h in roughly [0.7, 1.3])."""
    h = random_smooth(Nx, Ny, Lx, Ly, seed=seed, kmax=kmax, amp=h_amp, mean=1.0)
    vx = random_smooth(Nx, Ny, Lx, Ly, seed=seed + 1, kmax=kmax, amp=v_amp)
    vy = random_smooth(Nx, Ny, Lx, Ly, seed=seed + 2, kmax=kmax, amp=v_amp)
    sig = random_smooth(Nx, Ny, Lx, Ly, seed=seed + 3, kmax=kmax, amp=v_amp)
    return State(Nx, Ny, Lx, Ly, h=h, vx=vx, vy=vy, sigma=sig,
                 meta=dict(kind="random_state", seed=seed))


def _smooth_step(t: np.ndarray) -> np.ndarray:
    """C-infinity step: 0 for t <= 0, 1 for t >= 1, e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}) between."""
    t = np.clip(t, 0.0, 1.0)
    with np.errstate(divide="ignore", over="ignore"):
        a = np.where(t > 0.0, np.exp(-1.0 / np.where(t > 0.0, t, 1.0)), 0.0)
        b = np.where(t < 1.0, np.exp(-1.0 / np.where(t < 1.0, 1.0 - t, 1.0)), 0.0)
    return a / (a + b)


def crossing_solitons(N=4096, L=200.0, a=0.6, theta_deg=30.0, window=(0.35, 0.45)) -> State:
    """Two line solitary waves of amplitude a whose crests cross at the origin,
    rotated by +theta and -theta from the y axis (Section 5 crosses them at 90
    degrees; this is the rotated variant), on [-L/2, L/2)^2 with N^2 points.

    Soliton i has unit normal n_i = (cos theta_i, sin theta_i) and travelling
    coordinate xi_i = n_i . (x, y); it contributes its depth anomaly a sech^2
    (kappa xi_i) and its velocity profile v(xi_i) n_i of Eq. (sol). A line
    with an irrational slope is not periodic on the box, so both are tapered
    to zero in y by a C-infinity window w(y) (1 for |y| <= window[0] L, 0 for
    |y| >= window[1] L): the data are smooth and periodic.
        h = 1 + w(y) sum_i a sech^2(kappa xi_i),   v = w(y) sum_i v(xi_i) n_i.
    sigma starts at zero (no closed form).
    """
    sol = Soliton1D(a=a)
    x, y = coords(N, N, L, L)
    X, Y = x[None, :], y[:, None]
    y0, y1 = window[0] * L, window[1] * L
    w = 1.0 - _smooth_step((np.abs(Y) - y0) / (y1 - y0))
    h = np.ones((N, N))
    vx = np.zeros((N, N))
    vy = np.zeros((N, N))
    th = math.radians(theta_deg)
    for t in (th, -th):
        nx, ny = math.cos(t), math.sin(t)
        f = sol.fields(nx * X + ny * Y)
        h += w * (f["h"] - 1.0)
        vx += w * f["v"] * nx
        vy += w * f["v"] * ny
    return State(N, N, L, L, h=h, vx=vx, vy=vy, sigma=np.zeros((N, N)),
                 meta=dict(kind="crossing_solitons", a=a, theta_deg=theta_deg, window=window))


def random_band(Nx, Ny, Lx, Ly, seed=0, kx_max=60, ky_max=6, amp=0.2, mean=0.0) -> np.ndarray:
    """Seeded band-limited real field with separate mode limits per axis:
    mean + Re sum_{0 <= mx <= kx_max, |my| <= ky_max} c_m e^{i(mx X + my Y)},
    c_m = amp (p + i q) / (1 + mx^2 + my^2), p, q ~ N(0, 1), X, Y the
    coordinates scaled to [0, 2 pi). The sum is formed as the matrix product
    E_y C E_x^T of the coefficient matrix with the two exponential factors,
    so wide bands stay cheap on long axes."""
    rng = np.random.default_rng(seed)
    x, y = coords(Nx, Ny, Lx, Ly)
    X = 2 * math.pi * (x + 0.5 * Lx) / Lx
    Y = 2 * math.pi * (y + 0.5 * Ly) / Ly
    mxs = np.arange(0, min(kx_max, Nx // 2 - 1) + 1)
    kyl = min(ky_max, Ny // 2 - 1)
    mys = np.arange(-kyl, kyl + 1)
    MY, MX = np.meshgrid(mys, mxs, indexing="ij")
    C = amp * (rng.standard_normal(MX.shape) + 1j * rng.standard_normal(MX.shape)) / (1.0 + MX ** 2 + MY ** 2)
    C[(MX == 0) & (MY <= 0)] = 0.0
    Ey = np.exp(1j * np.outer(Y, mys))
    Ex = np.exp(1j * np.outer(X, mxs))
    return float(mean) + np.real(Ey @ C @ Ex.T)


def random_band_state(Nx, Ny, Lx, Ly, seed=0, kx_max=60, ky_max=6, h_amp=0.15, v_amp=0.1) -> State:
    """Seeded smooth positive depth and velocity from random_band fields."""
    f = lambda s, a, m=0.0: random_band(Nx, Ny, Lx, Ly, seed=seed + s, kx_max=kx_max, ky_max=ky_max, amp=a, mean=m)
    return State(Nx, Ny, Lx, Ly, h=f(0, h_amp, 1.0), vx=f(1, v_amp), vy=f(2, v_amp), sigma=f(3, v_amp),
                 meta=dict(kind="random_band_state", seed=seed))
