"""The benchmark's configuration against the oracle, at the kernel instantiations it times.

The headline runs precision 2 (FP32 passes, double-float refinement residual),
the polynomial GMRES start (guess 3) and one CUDA graph per RK4 step on a
2048 x 2048 grid, where every transform pass runs its length-2048 kernels
(the compile-time FP32 variants and the tensor-copied y-passes). Here:

* 8 RK4 steps of that configuration on 2048 x 64 and 64 x 2048 grids, so
  that the length-2048 x-passes and y-passes each meet the oracle's
  O.rk4_step (Section 3), element by element, at the mixed bar 1e-5 (relative
  L2 and maximum norm per field). The cubic start is in use from step 5 on.
* one right-hand side (Section 2.2 Eq. (1), Section 3) at the full 2048 x 2048
  size, on the benchmark's Gaussian hump carrying a smooth potential flow
  (so the nonlinear terms the FP32 passes form are not zero), in precision 0
  against O.rhs at 1e-10 and in precision 2 at 1e-5.

GMRES runs at the production tolerance 1e-10 on the GPU and at 1e-13 in the
oracle; two correct solvers then differ by about the condition number times
1e-10, far below both bars.
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


def relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# the benchmark's spacing dx = 100/2048 on both axes
THIN = [(2048, 64, 100.0, 3.125), (64, 2048, 3.125, 100.0)]


def thin_state(Nx, Ny, Lx, Ly, seed):
    """Band-limited smooth state: modes up to 60 along the 2048-point axis
    (wavenumbers up to 3.8, the Gaussian hump's band) and 6 along the short one."""
    kx, ky = (60, 6) if Nx >= Ny else (6, 60)
    return I.random_band_state(Nx, Ny, Lx, Ly, seed=seed, kx_max=kx, ky_max=ky)


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", THIN)
def test_headline_configuration_rk4_against_oracle(Nx, Ny, Lx, Ly):
    from paper_2306_09731_gb300.sgn import Solver
    dt, steps = 1e-3, 8
    st = thin_state(Nx, Ny, Lx, Ly, 31 * Nx + Ny)
    G = O.Grid(Nx, Ny, Lx, Ly)
    s = Solver(Nx, Ny, Lx, Ly, precision=2, guess=3, graph=1, tol=1e-10)
    s.autotune(3)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, dt, steps)
    stats = s.stats()
    s.close()
    ref = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, dt, steps, tol=1e-13)
    for x, r in zip(f[:3], ref[:3]):
        got = host(x)
        assert rel(got, r) < 1e-5
        assert relmax(got, r) < 1e-5
    assert stats["solves"] == 4 * steps
    assert stats["last_relres"] <= 1e-10


@pytest.fixture(scope="module")
def rhs_2048():
    st = I.gaussian_hump_flow(2048, 100.0, 0.5, 0.2)
    G = O.Grid(2048, 2048, 100.0, 100.0)
    ref = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    return st, ref


@pytest.mark.slow
@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (2, 1e-5)])
def test_rhs_2048_squared_against_oracle(rhs_2048, precision, bar):
    from paper_2306_09731_gb300.sgn import Solver
    st, (rht, rvxt, rvyt, rsg, info) = rhs_2048
    assert info["converged"]
    s = Solver(2048, 2048, 100.0, 100.0, precision=precision, tol=1e-12)
    sg = dev(st.sigma)
    ht, vxt, vyt = s.rhs(dev(st.h), dev(st.vx), dev(st.vy), sg)
    got = [host(x) for x in (ht, vxt, vyt)]
    s.close()
    for a, b in zip(got, (rht, rvxt, rvyt)):
        assert rel(a, b) < bar
    assert rel(host(sg), rsg) < (1e-10 if precision == 0 else 1e-8)
