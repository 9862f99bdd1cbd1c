"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types an oracle formula: each compares the oracle with a
closed form, a brute-force definition, a structural property or a number the
paper prints. ``test_planted_mistakes_are_caught`` shows that plausible slips
in the oracle (dropped term, wrong sign, swapped axes) fail at least one pin.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2306_09731_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ---------------------------------------------------------------- pin helpers
# Each returns an error figure; the tests bound it and the mutation test checks
# that a planted mistake pushes at least one figure past its bound.

def pin_trig_derivative():
    """Spectral derivative of a trigonometric polynomial is exact (Section 3)."""
    Nx, Ny, Lx, Ly = 32, 16, 7.0, 3.0
    G = O.Grid(Nx, Ny, Lx, Ly)
    X, Y = np.meshgrid(G.x, G.y)
    ax, ay = 2 * math.pi / Lx, 2 * math.pi / Ly
    f = np.cos(3 * ax * X + 2 * ay * Y) + 0.5 * np.sin(5 * ax * X - ay * Y)
    fx = -3 * ax * np.sin(3 * ax * X + 2 * ay * Y) + 2.5 * ax * np.cos(5 * ax * X - ay * Y)
    fy = -2 * ay * np.sin(3 * ax * X + 2 * ay * Y) - 0.5 * ay * np.cos(5 * ax * X - ay * Y)
    return max(np.abs(O.dx(G, f) - fx).max(), np.abs(O.dy(G, f) - fy).max())


def brute_dx(f, Lx, axis):
    """d/dx by explicit DFT sums (pure Python loops), Nyquist mode dropped."""
    f = np.asarray(f)
    if axis == 0:
        return brute_dx(f.T, Lx, 1).T
    Ny, Nx = f.shape
    out = np.zeros_like(f)
    for r in range(Ny):
        for n in range(Nx):
            s = 0.0 + 0.0j
            for k in range(Nx):
                m = k if k < Nx // 2 else k - Nx
                if k == Nx // 2:
                    continue
                Fk = sum(f[r, j] * complex(math.cos(2 * math.pi * k * j / Nx),
                                           -math.sin(2 * math.pi * k * j / Nx))
                         for j in range(Nx))
                s += 1j * (2 * math.pi * m / Lx) * Fk * complex(
                    math.cos(2 * math.pi * k * n / Nx), math.sin(2 * math.pi * k * n / Nx))
            out[r, n] = (s / Nx).real
    return out


def pin_bruteforce_dft():
    Nx, Ny, Lx, Ly = 8, 6, 2.5, 1.5
    G = O.Grid(Nx, Ny, Lx, Ly)
    f = np.random.default_rng(3).standard_normal((Ny, Nx))
    ex = brute_dx(f, Lx, 1)
    ey = brute_dx(f, Ly, 0)
    return max(np.abs(O.dx(G, f) - ex).max(), np.abs(O.dy(G, f) - ey).max())


def pin_manufactured_elliptic():
    """L[sigma] against a symbolic evaluation of Eq. (sigmav)'s left side."""
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y", real=True)
    Lx, Ly = 2 * math.pi, 4 * math.pi
    h = 1 + sp.Rational(3, 10) * sp.cos(x) * sp.sin(y / 2) + sp.Rational(1, 10) * sp.sin(2 * x)
    s = sp.sin(x) + sp.Rational(1, 2) * sp.cos(y) + sp.Rational(1, 5) * sp.sin(x + y / 2)
    L = 3 * s / h ** 3 - sp.diff(sp.diff(s, x) / h, x) - sp.diff(sp.diff(s, y) / h, y)
    fh, fs, fL = (sp.lambdify((x, y), e, "numpy") for e in (h, s, L))
    G = O.Grid(128, 128, Lx, Ly)
    X, Y = np.meshgrid(G.x, G.y)
    return rel(O.elliptic_apply(G, fh(X, Y), fs(X, Y)), fL(X, Y))


def pin_soliton_sigma():
    """GMRES solution of Eq. (sigmav) for the soliton vs sigma = m (h^2)'/6, Eq. (sol)."""
    st = I.soliton_256x16()
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    b = O.divergence_rhs(G, st.vx, st.vy)
    s, its, rr, conv = O.gmres(G, st.h, b, np.zeros_like(b), tol=1e-13)
    assert conv
    return rel(s, st.sigma)


def pin_soliton_rhs():
    """Travelling wave: (h, v)_t = -c d/dxi (h, v), v_y,t = 0 (Section 2.4)."""
    st = I.soliton_256x16()
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    f, c = st.meta["fields"], st.meta["c"]
    ht, vxt, vyt, _, _ = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    ones = np.ones((st.Ny, 1))
    return max(rel(ht, ones * (-c * f["h_xi"])), rel(vxt, ones * (-c * f["v_xi"])),
               float(np.abs(vyt).max()))


def pin_rk4_soliton():
    """100 RK4 steps of dt = 5e-3 against the exact soliton at t = 0.5."""
    st = I.soliton_256x16()
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    h, vx, vy, s = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, 5e-3, 100)
    ex = I.soliton_256x16(t=0.5)
    return max(rel(h, ex.h), rel(vx, ex.vx))


def pin_linear_dispersion():
    """h = 1 + eps cos(k x), v = 0 oscillates with omega^2 = g k^2 / (1 + k^2/3).

    Linearising Eqs. (1)-(3) about h = 1, v = 0 gives this relation (the
    Green-Naghdi linear dispersion); the O(eps^2) remainder is below the bound.
    """
    Nx, Ny, Lx, Ly = 32, 8, 2 * math.pi / 1.5, 1.0
    G = O.Grid(Nx, Ny, Lx, Ly)
    k = 2 * math.pi / Lx
    eps = 1e-6
    X = np.broadcast_to(G.x[None, :], (Ny, Nx))
    h = 1.0 + eps * np.cos(k * X)
    z = np.zeros((Ny, Nx))
    T, n = 1.0, 200
    hh, vx, vy, s = O.rk4_step(G, h, z, z, z, T / n, n, tol=1e-13)
    w = math.sqrt(k * k / (1 + k * k / 3))
    pred = 1.0 + eps * np.cos(k * X) * math.cos(w * T)
    return float(np.abs(hh - pred).max() / eps)


def pin_invariants_closed_form():
    """Mass, momentum and energy of the soliton against quadrature of Eq. (sol)."""
    quad = pytest.importorskip("scipy.integrate").quad
    st = I.soliton_256x16()
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    inv = O.invariants(G, st.h, st.vx, st.vy, st.sigma)
    sol = I.Soliton1D(a=0.5)
    c = sol.c

    def dens(x):
        f = sol.fields(np.array([x]))
        h, u, s = f["h"][0], f["u"][0], f["sigma"][0]
        return 0.5 * h * u * u + 1.5 * s * s / h ** 3 + 0.5 * (h - 1) ** 2

    mass = st.Ly * 2 * sol.a / sol.kappa
    energy = st.Ly * quad(dens, -40, 40, epsabs=1e-14, epsrel=1e-13, limit=200)[0]
    return max(abs(inv[0] - mass) / mass, abs(inv[1] - c * mass) / (c * mass),
               abs(inv[2]), abs(inv[3] - energy) / energy)


# ---------------------------------------------------------------------- tests

def test_grid_matches_paper_soliton_location():
    """Section 4.1 prints x_s = 6.995, a collocation point of the paper's grid."""
    gold = json.load(open(GOLDEN))["deformed_soliton_max"]
    G = O.Grid(gold["Nx"], gold["Ny"], gold["period_x"], gold["period_y"])
    assert np.min(np.abs(G.x - gold["x_s"])) < 5e-4
    assert G.x[0] == pytest.approx(-gold["period_x"] / 2)
    assert np.all(np.diff(G.x) > 0)


def test_trig_derivative_exact():
    assert pin_trig_derivative() < 1e-11


def test_derivative_matches_bruteforce_dft():
    assert pin_bruteforce_dft() < 1e-12


def test_elliptic_manufactured_solution():
    assert pin_manufactured_elliptic() < 1e-11


def test_elliptic_operator_symmetric_positive_definite():
    Nx, Ny = 8, 6
    G = O.Grid(Nx, Ny, 3.0, 2.0)
    h = I.random_smooth(Nx, Ny, 3.0, 2.0, seed=5, kmax=2, amp=0.2, mean=1.0)
    A = O.dense_elliptic_matrix(G, h)
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0.0


def test_preconditioner_is_operator_at_unit_depth():
    """M = L at h = 1 (Section 3), so GMRES converges in one iteration."""
    G = O.Grid(32, 16, 5.0, 3.0)
    s = I.random_smooth(32, 16, 5.0, 3.0, seed=1)
    h1 = np.ones_like(s)
    assert np.abs(O.precond_solve(G, O.elliptic_apply(G, h1, s)) - s).max() < 1e-13
    b = I.random_smooth(32, 16, 5.0, 3.0, seed=2)
    _, its, rr, conv = O.gmres(G, h1, b, np.zeros_like(b), tol=1e-12)
    assert conv and its == 1


def test_gmres_matches_dense_solve():
    Nx, Ny, Lx, Ly = 16, 8, 4.0, 2.0
    G = O.Grid(Nx, Ny, Lx, Ly)
    h = I.random_smooth(Nx, Ny, Lx, Ly, seed=7, kmax=3, amp=0.3, mean=1.0)
    b = I.random_smooth(Nx, Ny, Lx, Ly, seed=8, kmax=5)
    A = O.dense_elliptic_matrix(G, h)
    ref = np.linalg.solve(A, b.ravel()).reshape(Ny, Nx)
    s, its, rr, conv = O.gmres(G, h, b, np.zeros_like(b), tol=1e-13, restart=5)
    assert conv
    assert rel(s, ref) < 1e-11


def test_gmres_zero_rhs_and_restart_cap():
    G = O.Grid(16, 8, 4.0, 2.0)
    h = I.random_smooth(16, 8, 4.0, 2.0, seed=9, amp=0.3, mean=1.0)
    z = np.zeros_like(h)
    s, its, rr, conv = O.gmres(G, h, z, np.ones_like(h))
    assert conv and its == 0 and np.all(s == 0)
    b = I.random_smooth(16, 8, 4.0, 2.0, seed=10)
    s, its, rr, conv = O.gmres(G, h, b, z, tol=1e-15, restart=2, maxit=3)
    assert not conv and its == 3 and rr > 1e-15


def test_soliton_sigma_closed_form():
    assert pin_soliton_sigma() < 1e-9


def test_soliton_rhs_is_travelling_wave():
    assert pin_soliton_rhs() < 1e-8


def test_rk4_exact_soliton_256x16():
    """The line soliton workload: <= 1e-8 relative L2 from the exact solution at t = 0.5."""
    assert pin_rk4_soliton() < 1e-8


def test_rk4_fourth_order_in_time():
    st = I.line_soliton(128, 8, 40.0, 4.0, a=0.8)
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    errs = []
    T = 0.4
    for n in (4, 8):
        h, vx, vy, s = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, T / n, n, tol=1e-13)
        ex = I.line_soliton(128, 8, 40.0, 4.0, a=0.8, t=T)
        errs.append(rel(h, ex.h))
    order = math.log2(errs[0] / errs[1])
    assert 3.5 < order < 4.6, (errs, order)


def test_linear_dispersion_relation():
    assert pin_linear_dispersion() < 1e-5


def test_mass_conserved_and_curl_free():
    st = I.random_state(32, 32, 6.0, 6.0, seed=11)
    G = O.Grid(32, 32, 6.0, 6.0)
    # make v curl-free: v = grad(phi) for a smooth phi
    phi = I.random_smooth(32, 32, 6.0, 6.0, seed=12, kmax=4)
    vx, vy = O.dx(G, phi), O.dy(G, phi)
    m0 = O.invariants(G, st.h, vx, vy, np.zeros_like(vx))[0]
    h, vx2, vy2, s = O.rk4_step(G, st.h, vx, vy, np.zeros_like(vx), 2e-3, 5)
    m1 = O.invariants(G, h, vx2, vy2, s)[0]
    assert abs(m1 - m0) < 1e-12 * max(1.0, np.abs(st.h).sum() * G.dxdy)
    curl = O.dx(G, vy2) - O.dy(G, vx2)
    assert np.abs(curl).max() < 1e-11


def test_transpose_equivariance():
    """Swapping x and y (square box) transposes the result: catches axis mix-ups."""
    st = I.random_state(16, 16, 5.0, 5.0, seed=13)
    G = O.Grid(16, 16, 5.0, 5.0)
    a = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    b = O.rhs(G, st.h.T, st.vy.T, st.vx.T, st.sigma.T, tol=1e-13)
    assert np.abs(a[0] - b[0].T).max() < 1e-9
    assert np.abs(a[1] - b[2].T).max() < 1e-9
    assert np.abs(a[2] - b[1].T).max() < 1e-9


def test_energy_drift_soliton():
    st = I.soliton_256x16()
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    e0 = O.invariants(G, st.h, st.vx, st.vy, st.sigma)[3]
    h, vx, vy, s = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, 5e-3, 40)
    e1 = O.invariants(G, h, vx, vy, s)[3]
    assert abs(e1 - e0) / e0 < 1e-10


def test_invariants_closed_form():
    assert pin_invariants_closed_form() < 1e-9


def test_krasny_filter_zeroes_small_modes():
    Nx, Ny, Lx, Ly = 16, 8, 2 * math.pi, 2 * math.pi
    G = O.Grid(Nx, Ny, Lx, Ly)
    X, Y = np.meshgrid(G.x, G.y)
    f = 1.0 + 0.3 * np.cos(X) + 1e-14 * np.cos(3 * X + Y) + 1e-11 * np.sin(2 * Y)
    g = O.krasny(G, f, 1e-12)
    assert np.abs(g - (1.0 + 0.3 * np.cos(X) + 1e-11 * np.sin(2 * Y))).max() < 1e-15


def test_dealias_mask_two_thirds():
    G = O.Grid(12 * 2, 6 * 2, 1.0, 1.0)
    m = O.dealias_mask(G)
    kept_x = int(m[0].sum())
    kept_y = int(m[:, 0].sum())
    assert kept_x == 2 * (24 // 3) + 1 and kept_y == 2 * (12 // 3) + 1


def _rhs_cos_flow_closed_form(x, a, m, g=1.0):
    """Exact right-hand side for h = 1, vx = a cos(m x), vy = 0 on a 2 pi box.
    Eq. (sigmav) at h = 1 is 3 sigma - sigma_xx = a m sin(m x), so
    sigma = a m sin(m x)/(3 + m^2) and u = 3 a cos(m x)/(3 + m^2):
    h_t = 3 a m sin(m x)/(3 + m^2) (mode m). F = |v|^2/2 - sigma_x^2/2 + g -
    9 sigma^2/2 is a constant plus A cos(2 m x) with
    A = (a^2/4)(1 - (m^4 - 9 m^2)/(3 + m^2)^2), so vx_t = 2 m A sin(2 m x)
    (mode 2m, the only one the products create)."""
    ht = 3.0 * a * m * np.sin(m * x) / (3.0 + m * m)
    A = 0.25 * a * a * (1.0 - (m ** 4 - 9.0 * m * m) / (3.0 + m * m) ** 2)
    return ht, 2.0 * m * A * np.sin(2 * m * x)


def pin_dealias_closed_form():
    """The 2/3 rule on the right-hand side (dealias=True): on 32 points the
    product mode 2m = 12 has 3|m| = 36 > 32 and must vanish from vx_t while
    h_t (mode 6) is unchanged; on 30 points mode 10 has 3|m| = 30 <= 30 and
    must stay; without the rule mode 12 is there. Largest error against the
    closed forms."""
    a, err = 0.3, 0.0
    for Nx, m, dealias, keep in ((32, 6, True, False), (30, 5, True, True), (32, 6, False, True)):
        G = O.Grid(Nx, 4, 2 * math.pi, 2 * math.pi)
        X = np.broadcast_to(G.x[None, :], (4, Nx))
        vx = a * np.cos(m * X)
        z = np.zeros_like(vx)
        ht, vxt, vyt, _, _ = O.rhs(G, np.ones_like(vx), vx, z, z, tol=1e-14, dealias=dealias)
        eht, evxt = _rhs_cos_flow_closed_form(X, a, m)
        err = max(err, np.abs(ht - eht).max(), np.abs(vxt - (evxt if keep else 0.0)).max(), np.abs(vyt).max())
        assert np.abs(evxt).max() > 1e-3  # the product mode is present in the exact RHS
    return err


def test_dealias_rhs_closed_form():
    assert pin_dealias_closed_form() < 1e-13


# --------------------------------------------------------- planted mistakes

MUTANTS = {}


def _mutant(name):
    def deco(fn):
        MUTANTS[name] = fn
        return fn
    return deco


@_mutant("drop_3sigma_over_h3")
def _m1(monkeypatch):
    monkeypatch.setattr(O, "elliptic_apply",
                        lambda G, h, s: -O.dx(G, O.dx(G, s) / h) - O.dy(G, O.dy(G, s) / h))


@_mutant("wrong_sign_sigma_squared_term")
def _m2(monkeypatch):
    orig = O.rhs

    def bad(G, h, vx, vy, sigma0, g=1.0, **kw):
        ht, vxt, vyt, s, info = orig(G, h, vx, vy, sigma0, g=g, **kw)
        corr = 9.0 * s ** 2 / h ** 4  # flips -9/2 sigma^2/h^4 to +9/2
        return ht, vxt - O.dx(G, corr), vyt - O.dy(G, corr), s, info
    monkeypatch.setattr(O, "rhs", bad)


@_mutant("swapped_wavenumber_axes")
def _m3(monkeypatch):
    orig = O.Grid.__init__

    def init(self, Nx, Ny, Lx, Ly):
        orig(self, Nx, Ny, Lx, Ly)
        kx = np.fft.fftfreq(Nx, d=1.0 / Nx) * 2 * math.pi / Ly
        kx[Nx // 2] = 0
        self.KX = kx[None, :]
    monkeypatch.setattr(O.Grid, "__init__", init)


@_mutant("h_instead_of_inverse_h_in_flux")
def _m4(monkeypatch):
    monkeypatch.setattr(O, "elliptic_apply",
                        lambda G, h, s: 3 * s / h ** 3 - O.dx(G, O.dx(G, s) * h) - O.dy(G, O.dy(G, s) * h))


@_mutant("rk4_wrong_weights")
def _m5(monkeypatch):
    orig = O.rhs
    state = {"n": 0}

    def bad(*a, **kw):
        out = orig(*a, **kw)
        state["n"] += 1
        if state["n"] % 4 == 2:  # stage 2 weight effectively 1 instead of 2
            return (0.5 * out[0], 0.5 * out[1], 0.5 * out[2]) + out[3:]
        return out
    monkeypatch.setattr(O, "rhs", bad)


@_mutant("dealias_mask_skipped")
def _m7(monkeypatch):
    monkeypatch.setattr(O, "dealias_mask", lambda G: np.ones((G.Ny, G.Nx)))


@_mutant("dealias_strict_inequality")
def _m8(monkeypatch):
    def strict(G):
        keep_x = 3.0 * np.abs(G.mx) < G.Nx
        keep_y = 3.0 * np.abs(G.my) < G.Ny
        return (keep_y[:, None] & keep_x[None, :]).astype(np.float64)
    monkeypatch.setattr(O, "dealias_mask", strict)


@_mutant("missing_gravity_term")
def _m6(monkeypatch):
    orig = O.rhs

    def bad(G, h, vx, vy, sigma0, g=1.0, **kw):
        return orig(G, h, vx, vy, sigma0, g=0.0, **kw)
    monkeypatch.setattr(O, "rhs", bad)


PINS = [(pin_trig_derivative, 1e-11), (pin_manufactured_elliptic, 1e-11),
        (pin_soliton_sigma, 1e-9), (pin_soliton_rhs, 1e-8), (pin_rk4_soliton, 1e-8),
        (pin_linear_dispersion, 1e-5), (pin_dealias_closed_form, 1e-13)]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistakes_are_caught(name, monkeypatch):
    pytest.importorskip("sympy")
    MUTANTS[name](monkeypatch)
    failed = []
    for fn, bound in PINS:
        try:
            err = fn()
        except (AssertionError, FloatingPointError, np.linalg.LinAlgError, ZeroDivisionError):
            err = float("inf")
        if not (err < bound):
            failed.append(fn.__name__)
            break
    assert failed, f"mutant {name} passed every pin"


# ----------------------------------------------------------- diagnostics
# Pins of oracle.diagnostics (Sections 3, 4.1, 4.2) against closed forms.

def test_diagnostics_exact_soliton_closed_form():
    """An exact line solitary wave centred on a grid point: crest at that point,
    c from the crest equals the wave's speed, no deviation, vy = 0."""
    G = O.Grid(256, 8, 80.0, 4.0)
    j0 = 141
    st = I.line_soliton(256, 8, 80.0, 4.0, a=0.5, x0=float(G.x[j0]))
    d = O.diagnostics(G, st.h, st.vx, st.vy)
    assert d["i_max"] == j0 and d["x_s"] == float(G.x[j0]) and d["y_s"] == float(G.y[0])
    assert d["h_max"] == 1.5
    assert abs(d["c_fit"] - I.Soliton1D(a=0.5).c) < 1e-15
    assert d["dev_h"] < 1e-14 and d["dev_vx"] < 1e-13 and d["max_vy"] == 0.0


def test_diagnostics_soliton_shifted_by_half_a_cell():
    """A crest between grid points: the maximum sits on the nearer point and the
    deviation is the closed-form difference between the two centres."""
    G = O.Grid(512, 4, 80.0, 2.0)
    j0 = 300
    x0 = float(G.x[j0]) + 0.3 * G.Lx / G.Nx
    st = I.line_soliton(512, 4, 80.0, 2.0, a=0.4, x0=x0)
    d = O.diagnostics(G, st.h, st.vx, st.vy)
    assert d["i_max"] == j0
    sol = I.Soliton1D(a=d["h_max"] - 1.0)
    xi = G.x - d["x_s"]
    ref = np.max(np.abs(st.h[0] - sol.fields(xi)["h"]))
    assert abs(d["dev_h"] - ref) < 1e-14 and d["dev_h"] > 1e-4


def test_diagnostics_tail_of_single_modes():
    """cos(m x): one DFT pair of size N/2 each, so the monitor reads 1/2 when m
    lies in the outer band (16 m >= 7 N) and rounding level otherwise."""
    G = O.Grid(64, 32, 2 * np.pi, 2 * np.pi)
    X = np.broadcast_to(G.x[None, :], (32, 64))
    Y = np.broadcast_to(G.y[:, None], (32, 64))
    one = np.ones((32, 64))
    d = O.diagnostics(G, one + 0.1 * np.cos(29 * X), np.cos(10 * X), np.sin(15 * Y))
    assert abs(d["tail"][0] - 0.05) < 1e-15
    assert d["tail"][1] < 1e-15
    assert abs(d["tail"][2] - 0.5) < 1e-15


def test_diagnostics_ties_and_no_crest():
    G = O.Grid(16, 8, 4.0, 2.0)
    h = np.ones((8, 16))
    h[3, 5] = 1.2
    h[2, 9] = 1.2
    d = O.diagnostics(G, h, np.zeros_like(h), np.zeros_like(h))
    assert d["i_max"] == 2 * 16 + 9 and d["h_max"] == 1.2
    flat = O.diagnostics(G, np.ones((8, 16)), np.zeros((8, 16)), np.zeros((8, 16)))
    assert flat["i_max"] == 0 and np.isnan(flat["dev_h"]) and np.isnan(flat["dev_vx"])


# ------------------------------------------- coarse transfer of the learned start

def test_coarse_sample_of_band_limited_field_is_point_sampling():
    G = O.Grid(64, 32, 6.0, 3.0)
    X = np.broadcast_to(G.x[None, :], (32, 64))
    Y = np.broadcast_to(G.y[:, None], (32, 64))
    kx, ky = 2 * np.pi / 6.0, 2 * np.pi / 3.0
    f = 1.0 + 0.5 * np.cos(3 * kx * X) * np.sin(2 * ky * Y) + 0.2 * np.sin(7 * kx * X)
    c = O.coarse_sample(G, f, 16)
    assert np.max(np.abs(c - f[::2, ::4])) < 1e-13
    # modes at or above n/2 = 8 vanish from the samples
    g = np.cos(8 * kx * X) + np.sin(9 * ky * Y)
    assert np.max(np.abs(O.coarse_sample(G, g, 16))) < 1e-13


def test_coarse_embed_is_band_limited_interpolation():
    G = O.Grid(64, 64, 2 * np.pi, 2 * np.pi)
    i = np.arange(16)
    fc = np.cos(2 * np.pi * 3 * i[None, :] / 16) * np.ones((16, 1)) + 0.5 * np.sin(2 * np.pi * 5 * i[:, None] / 16)
    f = O.coarse_embed(G, fc, 16, scale=2.0)
    X = np.broadcast_to(G.x[None, :] - G.x[0], (64, 64))
    Y = np.broadcast_to(G.y[:, None] - G.y[0], (64, 64))
    ref = 2.0 * (np.cos(3 * X) + 0.5 * np.sin(5 * Y))
    assert np.max(np.abs(f - ref)) < 1e-13
    assert np.max(np.abs(O.coarse_sample(G, f, 16) - 2.0 * fc)) < 1e-13
