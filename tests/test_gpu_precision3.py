"""Precision 3: the inner GMRES in FP32, everything else of the RK4 stage in
double-float (the refinement matvec, the coefficients, the right-hand side
and its K spectra) or FP64 (state, dots, Givens, residual).

Bars: the FP64 path's. Right-hand side within 1e-10 relative L2 of the FP64
oracle: the double-float unit roundoff 2^-48, grown by the log2 N stages of
the transforms and the wavenumbers of the derivatives (~100 on these grids),
stays near 1e-12. RK4 fields within 1e-10 of the oracle (every solve at
tol = 1e-12); the line soliton within 1e-8 of the exact solution; graph mode
bitwise equal to the host loop; and on the transverse-stability workload at a
= 1 (where precision 1's FP32 right-hand side seeds growing modes) within 1e-9
of the FP64 path after 250 steps.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2306_09731_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def solver(*a, **kw):
    from paper_2306_09731_gb300.sgn import Solver
    return Solver(*a, precision=3, **kw)


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", [(64, 32, 8.0, 5.0), (256, 16, 80.0, 10.0), (128, 128, 10.0, 10.0),
                                         (512, 1024, 40.0, 60.0)])
def test_p3_rhs_parity(Nx, Ny, Lx, Ly):
    st = I.random_state(Nx, Ny, Lx, Ly, seed=Nx + 13 * Ny)
    G = O.Grid(Nx, Ny, Lx, Ly)
    s = solver(Nx, Ny, Lx, Ly, tol=1e-12)
    sg = dev(st.sigma)
    ht, vxt, vyt = s.rhs(dev(st.h), dev(st.vx), dev(st.vy), sg)
    rht, rvxt, rvyt, rsg, _ = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    for a, b in ((ht, rht), (vxt, rvxt), (vyt, rvyt)):
        assert rel(host(a), b) < 1e-10
    s.close()


def test_p3_rk4_random_against_oracle():
    Nx, Ny, L = 64, 64, 8.0
    st = I.random_state(Nx, Ny, L, L, seed=31)
    G = O.Grid(Nx, Ny, L, L)
    phi = I.random_smooth(Nx, Ny, L, L, seed=32, kmax=4)
    vx, vy = O.dx(G, phi), O.dy(G, phi)
    z = np.zeros_like(vx)
    s = solver(Nx, Ny, L, L, dealias=1, tol=1e-12)
    a = [dev(st.h), dev(vx), dev(vy), dev(z)]
    s.rk4_step(*a, 2e-3, 8)
    ref = O.rk4_step(G, st.h, vx, vy, z, 2e-3, 8, tol=1e-13, dealias=True)
    for x, r in zip(a[:3], ref[:3]):
        assert rel(host(x), r) < 1e-10
    s.close()


def test_p3_soliton_against_exact_and_graph_bitwise():
    st = I.soliton_256x16()
    out = {}
    for graph in (1, 0):
        s = solver(st.Nx, st.Ny, st.Lx, st.Ly, guess=2, graph=graph)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        s.rk4_step(*f, 5e-3, 100)
        out[graph] = ([host(x) for x in f], s.stats())
        s.close()
    ex = I.soliton_256x16(t=0.5)
    assert rel(out[1][0][0], ex.h) < 1e-8 and rel(out[1][0][1], ex.vx) < 1e-8
    for x, y in zip(out[1][0], out[0][0]):
        assert np.array_equal(x, y)
    assert out[1][1]["matvecs"] == out[0][1]["matvecs"]


def test_p3_follows_fp64_where_precision1_drifts():
    from paper_2306_09731_gb300.sgn import Solver
    st = I.perturbed_soliton(1024, 256, 120.0, 30.0, a=1.0, eps=1e-2, seed=0)
    res = {}
    for prec in (0, 3):
        s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, precision=prec, guess=2, graph=1)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        s.rk4_step(*f, 2e-3, 250)
        res[prec] = [host(x) for x in f[:3]]
        s.close()
    (h3, vx3, vy3), (h0, vx0, vy0) = res[3], res[0]
    vnorm = np.sqrt(np.linalg.norm(vx0) ** 2 + np.linalg.norm(vy0) ** 2)
    assert rel(h3, h0) < 1e-9
    assert np.linalg.norm(vx3 - vx0) < 1e-9 * vnorm
    assert np.linalg.norm(vy3 - vy0) < 1e-9 * vnorm
