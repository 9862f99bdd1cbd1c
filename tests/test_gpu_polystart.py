"""The polynomial start across steps (guess = 3).

Each RK4 stage starts GMRES from the polynomial in time through the same
stage's sigma at the last 3 (quadratic) or 4 (cubic) steps; until the handle
has 3 steps of the trajectory it starts as guess 2 does. Only GMRES's starting
value changes, so the bars are those of every other start: the FP64 oracle
within 1e-10 (FP64 path) and 1e-5 (the FP32 bulk), graph mode bitwise equal to
the host loop, and, once the history is built, fewer matvecs than guess 2.
With the FP32 right-hand side the start relies on the update adding the
right-hand side's linear part in FP64: FP32 rounding of the whole would enter
sigma as step-to-step noise that the cubic amplifies.
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


STAT_KEYS = ("matvecs", "solves", "max_iters", "last_iters", "last_relres", "refinements")


def run(st, graph, steps, dt, **opts):
    from paper_2306_09731_gb300.sgn import Solver
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, graph=graph, **opts)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, dt, steps)
    out = [host(x) for x in f]
    stats = s.stats()
    s.close()
    return out, stats


@pytest.mark.parametrize("precision", [0, 2, 3])
def test_poly_start_graph_matches_host_loop_bitwise(precision):
    st = I.perturbed_soliton(256, 64, 60.0, 15.0, a=0.5, eps=5e-2, seed=3)
    a, sa = run(st, 1, 8, 2e-3, precision=precision, guess=3)
    b, sb = run(st, 0, 8, 2e-3, precision=precision, guess=3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for k in STAT_KEYS:
        assert sa[k] == sb[k], k
    assert sa["solves"] == 32


def oracle_case():
    Nx, Ny, L = 64, 64, 8.0
    st = I.random_state(Nx, Ny, L, L, seed=31)
    G = O.Grid(Nx, Ny, L, L)
    phi = I.random_smooth(Nx, Ny, L, L, seed=32, kmax=4)
    vx, vy = O.dx(G, phi), O.dy(G, phi)
    return G, st.h, vx, vy, np.zeros_like(vx)


@pytest.mark.parametrize("precision,graph,bar", [(0, 0, 1e-10), (0, 1, 1e-10), (2, 1, 1e-5)])
def test_poly_start_parity_with_oracle(precision, graph, bar):
    """Eight steps (the cubic start runs from step 5 on) against the oracle,
    which starts every solve from the last sigma."""
    from paper_2306_09731_gb300.sgn import Solver
    G, h, vx, vy, z = oracle_case()
    tol = 1e-12 if precision == 0 else 1e-10
    s = Solver(G.Nx, G.Ny, G.Lx, G.Ly, precision=precision, guess=3, graph=graph, dealias=1, tol=tol)
    a = [dev(h), dev(vx), dev(vy), dev(z)]
    s.rk4_step(*a, 2e-3, 8)
    ref = O.rk4_step(G, h, vx, vy, z, 2e-3, 8, tol=1e-13, dealias=True)
    for x, r in zip(a[:3], ref[:3]):
        assert rel(host(x), r) < bar
    s.close()


@pytest.mark.parametrize("precision", [0, 2, 3])
def test_poly_start_fewer_matvecs_than_linear(precision):
    """Once 4 steps are held the cubic start leaves far less for GMRES to do
    than guess 2's linear extrapolation inside a step; the trajectories agree
    to the path's bar."""
    from paper_2306_09731_gb300.sgn import Solver
    st = I.gaussian_hump(256, 25.0, 0.5)
    per, fields = {}, {}
    for guess in (2, 3):
        s = Solver(256, 256, 25.0, 25.0, precision=precision, guess=guess, graph=1)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        s.rk4_step(*f, 1e-3, 4)
        m0 = s.stats()["matvecs"]
        s.rk4_step(*f, 1e-3, 8)
        st1 = s.stats()
        per[guess] = st1["matvecs"] - m0
        assert st1["max_iters"] < 1000
        fields[guess] = [host(x) for x in f[:3]]
        s.close()
    assert per[3] <= 0.6 * per[2], per
    bar = 1e-9 if precision != 2 else 1e-6
    for x, y in zip(fields[3], fields[2]):
        assert rel(x, y) < bar


@pytest.mark.parametrize("graph", [0, 1])
def test_poly_start_history_across_calls(graph):
    """A call that continues the trajectory keeps the ring of past steps
    (fewer matvecs than a fresh handle on the same input); a call on another
    state starts without it, bitwise equal to a fresh handle."""
    from paper_2306_09731_gb300.sgn import Solver
    st = I.gaussian_hump(256, 25.0, 0.5)
    mk = lambda: Solver(256, 256, 25.0, 25.0, precision=2, guess=3, graph=graph)
    a = mk()
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    a.rk4_step(*f, 1e-3, 4)
    mid = [host(x).copy() for x in f]
    m0 = a.stats()["matvecs"]
    a.rk4_step(*f, 1e-3, 1)
    cont = a.stats()["matvecs"] - m0
    b = mk()
    g = [dev(x) for x in mid]
    b.rk4_step(*g, 1e-3, 1)
    fresh = b.stats()["matvecs"]
    assert cont < fresh
    for x, y in zip(f[:3], g[:3]):
        assert rel(host(x), host(y)) < 1e-6
    pert = [x.copy() for x in mid]
    pert[0] = pert[0] + 1e-3 * np.cos(np.linspace(0.0, 2.0 * np.pi, 256))[None, :]
    # five steps: the quadratic and the cubic start read only steps of this call
    p1 = [dev(x) for x in pert]
    a.rk4_step(*p1, 1e-3, 5)
    c = mk()
    p2 = [dev(x) for x in pert]
    c.rk4_step(*p2, 1e-3, 5)
    for x, y in zip(p1, p2):
        assert np.array_equal(host(x), host(y))
    for s in (a, b, c):
        s.close()


def test_poly_start_records_only_once_the_start_is_cubic():
    """The learned start corrects the polynomial start only once the ring holds
    4 steps of the trajectory: a call of 4 steps from a fresh history records
    nothing, one of 6 steps all four stages of its last 2 (every call other
    than an RK4 step, sgn_record_learned included, restarts the history)."""
    from paper_2306_09731_gb300.sgn import Solver
    st = I.gaussian_hump(64, 8.0, 0.5)
    for steps, expect in ((4, 0), (6, 8)):
        s = Solver(64, 64, 8.0, 8.0, precision=2, guess=3)
        f = [dev(a) for a in (st.h, st.vx, st.vy, st.sigma)]
        s.record_learned(16, 32)
        s.rk4_step(*f, 1e-3, steps)
        assert s.stop_recording() == expect
        s.close()
