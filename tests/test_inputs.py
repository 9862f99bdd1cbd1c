"""Host checks of the seeded workload generators that have no closed-form pin
elsewhere: the rotated crossing solitons and the band-limited random fields."""
import math

import numpy as np

from paper_2306_09731_gb300 import inputs as I


def test_crossing_solitons_shape_symmetry_and_limits():
    st = I.crossing_solitons(256, 200.0, 0.6, 30.0)
    # crests cross at the origin: h = 1 + 2a there (the window is 1 near y = 0)
    x, y = I.coords(256, 256, 200.0, 200.0)
    i0, j0 = int(np.argmin(np.abs(y))), int(np.argmin(np.abs(x)))
    assert abs(st.h[i0, j0] - 2.2) < 1e-12
    # the +theta / -theta pair is mirror symmetric in y: h, vx even, vy odd
    # (row l <-> row N - l about y = 0 on the grid y_l = -L/2 + l L/N)
    flip = lambda f: np.roll(f[::-1], 1, axis=0)
    assert np.allclose(st.h, flip(st.h), atol=1e-13)
    assert np.allclose(st.vx, flip(st.vx), atol=1e-13)
    assert np.allclose(st.vy, -flip(st.vy), atol=1e-13)
    # far from both crests and outside the window the data are at rest
    assert abs(st.h[0, 0] - 1.0) < 1e-14 and abs(st.vx[0, 0]) < 1e-14


def test_crossing_solitons_reduce_to_the_line_soliton_at_theta_zero():
    """theta = 0: both crests on x = 0, so inside the window the depth anomaly
    and v_x are twice those of one line soliton of Eq. (sol), v_y = 0."""
    st = I.crossing_solitons(128, 100.0, 0.5, 0.0, window=(0.4, 0.49))
    line = I.line_soliton(128, 128, 100.0, 100.0, a=0.5)
    x, y = I.coords(128, 128, 100.0, 100.0)
    rows = np.abs(y) <= 0.4 * 100.0
    assert np.allclose(st.h[rows] - 1.0, 2.0 * (line.h[rows] - 1.0), atol=1e-14)
    assert np.allclose(st.vx[rows], 2.0 * line.vx[rows], atol=1e-14)
    assert np.max(np.abs(st.vy)) == 0.0


def test_crossing_solitons_are_smooth_and_periodic():
    """At the benchmark's spacing (0.049) and half its box (the taper then
    spans 10 length units): the Fourier tail of every field is at rounding
    level, so the taper leaves no jump at the box edge."""
    st = I.crossing_solitons(2048, 100.0, 0.6, 15.0)
    for f in (st.h - 1.0, st.vx, st.vy):
        F = np.abs(np.fft.rfft2(f))
        tail = max(F[768:1280, :].max(), F[:, 768:].max())
        assert tail < 1e-12 * F.max()


def test_random_band_matches_its_sum():
    """The matrix-product form equals the double sum of its definition."""
    Nx, Ny, Lx, Ly = 16, 8, 3.0, 2.0
    f = I.random_band(Nx, Ny, Lx, Ly, seed=4, kx_max=5, ky_max=2, amp=0.3, mean=1.0)
    rng = np.random.default_rng(4)
    mxs, mys = np.arange(0, 6), np.arange(-2, 3)
    P = rng.standard_normal((len(mys), len(mxs)))
    Q = rng.standard_normal((len(mys), len(mxs)))
    x, y = I.coords(Nx, Ny, Lx, Ly)
    X = 2 * math.pi * (x + 0.5 * Lx) / Lx
    Y = 2 * math.pi * (y + 0.5 * Ly) / Ly
    ref = np.ones((Ny, Nx))
    for a, my in enumerate(mys):
        for b, mx in enumerate(mxs):
            if mx == 0 and my <= 0:
                continue
            w = 0.3 / (1.0 + mx * mx + my * my)
            ph = mx * X[None, :] + my * Y[:, None]
            ref += w * (P[a, b] * np.cos(ph) - Q[a, b] * np.sin(ph))
    assert np.max(np.abs(f - ref)) < 1e-13


def test_gaussian_hump_flow_is_curl_free_potential_flow():
    """v = grad(phi) of the stated potential: compared with a centred finite
    difference of phi, and curl v = 0 by the same differences."""
    from paper_2306_09731_gb300 import inputs as I
    N, L, beta = 256, 20.0, 0.2
    st = I.gaussian_hump_flow(N, L, 0.5, beta)
    x, y = I.coords(N, N, L, L)
    d = 1e-5
    phi = lambda X, Y: beta * np.exp(-0.5 * ((X - 1.0) ** 2 + Y ** 2))
    X, Y = np.meshgrid(x, y)
    assert np.abs(st.vx - (phi(X + d, Y) - phi(X - d, Y)) / (2 * d)).max() < 1e-9
    assert np.abs(st.vy - (phi(X, Y + d) - phi(X, Y - d)) / (2 * d)).max() < 1e-9
    assert np.abs(st.h - 1.0 - 0.5 * np.exp(-(X ** 2 + Y ** 2))).max() < 1e-15
    assert not st.sigma.any()
