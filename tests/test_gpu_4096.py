"""4096-point axes: the passes whose transforms take 512 threads (one column
or row pair per block in every type).

Bars are those of the smaller grids: FP64 operator and fields within 1e-10 of
the oracle (1e-12 for one application of L), double-float L within 1e-11,
FP32-bulk RK4 fields within 1e-5 (precision 3, whose right-hand side is
double-float: 1e-10), every GMRES solve at the FP64 tolerance. The
FP32 RHS meets 1e-5 as well: its terms linear in the state are added in FP64,
so its FP32 rounding scales with the nonlinear part only. Thin grids (4096 x
16, 16 x 4096, 4096 x 64) keep the oracle fast and put the 4096-point
transforms on each axis in turn; the crossing-soliton workload at 4096^2
checks the full-size operator against the oracle and two RK4 steps of the
mixed path against the FP64 path.
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
    return Solver(*a, **kw)


THIN = [(4096, 16, 200.0, 4.0), (16, 4096, 4.0, 200.0), (4096, 64, 300.0, 10.0)]


def thin_state(Nx, Ny, Lx, Ly, seed):
    """Random smooth state with modes up to 60 along the long axis and 6 along
    the short one (6 along a 4096-point axis would over-resolve it 340 times,
    and the FP32 derivative noise grows with that ratio)."""
    kx, ky = (60, 6) if Nx >= Ny else (6, 60)
    return I.random_band_state(Nx, Ny, Lx, Ly, seed=seed, kx_max=kx, ky_max=ky)


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", THIN)
@pytest.mark.parametrize("precision,bar", [(0, 1e-12), (2, 1e-11)])
def test_elliptic_apply_4096(Nx, Ny, Lx, Ly, precision, bar):
    st = thin_state(Nx, Ny, Lx, Ly, Nx + Ny)
    s = solver(Nx, Ny, Lx, Ly, precision=precision)
    out = host(s.elliptic_apply(dev(st.h), dev(st.sigma)))
    ref = O.elliptic_apply(O.Grid(Nx, Ny, Lx, Ly), st.h, st.sigma)
    assert rel(out, ref) < bar
    s.close()


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", THIN)
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_gmres_4096_meets_fp64_tolerance(Nx, Ny, Lx, Ly, precision):
    tol = 1e-10
    st = thin_state(Nx, Ny, Lx, Ly, 3 * Nx + Ny)
    G = O.Grid(Nx, Ny, Lx, Ly)
    b = O.divergence_rhs(G, st.vx, st.vy)
    s = solver(Nx, Ny, Lx, Ly, precision=precision, tol=tol)
    sig, its, rr, conv = s.gmres_solve(dev(st.h), dev(b), dev(np.zeros_like(b)))
    assert conv and rr <= tol
    c = O.precond_solve(G, b)
    r = c - O.precond_solve(G, O.elliptic_apply(G, st.h, host(sig)))
    assert np.linalg.norm(r) / np.linalg.norm(c) <= 2 * tol
    s.close()


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", THIN[:2])
@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (1, 1e-5), (2, 1e-5), (3, 1e-10)])
def test_rhs_4096(Nx, Ny, Lx, Ly, precision, bar):
    st = thin_state(Nx, Ny, Lx, Ly, Nx + 5 * Ny)
    G = O.Grid(Nx, Ny, Lx, Ly)
    s = solver(Nx, Ny, Lx, Ly, precision=precision, tol=1e-12)
    sg = dev(st.sigma)
    ht, vxt, vyt = s.rhs(dev(st.h), dev(st.vx), dev(st.vy), sg)
    rht, rvxt, rvyt, rsg, _ = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    errs = [rel(host(a), b) for a, b in ((ht, rht), (vxt, rvxt), (vyt, rvyt))]
    assert max(errs) < bar, errs
    s.close()


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", THIN[:2])
@pytest.mark.parametrize("precision,graph,bar", [(0, 0, 1e-10), (0, 1, 1e-10), (2, 1, 1e-5), (3, 1, 1e-10)])
def test_rk4_4096_against_oracle(Nx, Ny, Lx, Ly, precision, graph, bar):
    st = thin_state(Nx, Ny, Lx, Ly, 7 * Nx + Ny)
    G = O.Grid(Nx, Ny, Lx, Ly)
    s = solver(Nx, Ny, Lx, Ly, precision=precision, graph=graph, guess=2, tol=1e-12)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, 2e-3, 2)
    ref = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, 2e-3, 2, tol=1e-13)
    for x, r in zip(f[:3], ref[:3]):
        assert rel(host(x), r) < bar
    s.close()


def test_crossing_solitons_4096_squared():
    """The 4096^2 workload: the double-float operator against the oracle at full
    size, then two RK4 steps of precision 2 (graph mode) against the FP64 path;
    mass is conserved by both."""
    st = I.crossing_solitons(4096, 200.0, 0.6, 30.0)
    X, Y = np.meshgrid(*I.coords(4096, 4096, 200.0, 200.0))
    sig = 0.3 * np.exp(-0.01 * (X ** 2 + Y ** 2)) * np.cos(0.7 * X)
    s = solver(4096, 4096, 200.0, 200.0, precision=2)
    out = host(s.elliptic_apply(dev(st.h), dev(sig)))
    s.close()
    ref = O.elliptic_apply(O.Grid(4096, 4096, 200.0, 200.0), st.h, sig)
    assert rel(out, ref) < 1e-11
    del out, ref, X, Y, sig
    runs = {}
    for prec, graph in ((2, 1), (0, 0)):
        s = solver(4096, 4096, 200.0, 200.0, precision=prec, guess=2, graph=graph)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        m0 = s.invariants(*f)[0]
        s.rk4_step(*f, 1e-3, 2)
        m1 = s.invariants(*f)[0]
        assert abs(m1 - m0) < 1e-13 * 200.0 * 200.0
        assert s.stats()["solves"] == 8
        runs[prec] = [host(x) for x in f[:3]]
        s.close()
        del f
        torch.cuda.empty_cache()
    for a, b in zip(runs[2], runs[0]):
        assert rel(a, b) < 1e-5
