"""Graph mode (graph = 1): one RK4 step replayed as a CUDA graph whose GMRES
restart cycles and Arnoldi steps are conditional WHILE nodes, with the host
loop's stopping tests taken by device-side control kernels.

The kernels and their arithmetic are those of the host-driven loop, and every
reduction is deterministic, so the bar is bitwise equality with the host loop
(fields and GMRES statistics), plus the oracle bars of the FP64 path.
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


def run(st, graph, steps, dt, **opts):
    """Fields after `steps` RK4 steps and the handle's statistics."""
    from paper_2306_09731_gb300.sgn import Solver
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, graph=graph, **opts)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, dt, steps)
    out = [host(x) for x in f]
    stats = s.stats()
    s.close()
    return out, stats


STAT_KEYS = ("matvecs", "solves", "max_iters", "last_iters", "last_relres", "refinements")


@pytest.mark.parametrize("precision,guess", [(0, 0), (0, 2), (1, 0), (1, 2), (2, 2), (3, 2)])
def test_graph_matches_host_loop_bitwise(precision, guess):
    st = I.perturbed_soliton(256, 64, 60.0, 15.0, a=0.5, eps=5e-2, seed=3)
    a, sa = run(st, 1, 6, 2e-3, precision=precision, guess=guess)
    b, sb = run(st, 0, 6, 2e-3, precision=precision, guess=guess)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for k in STAT_KEYS:
        assert sa[k] == sb[k], k
    assert sa["solves"] == 24


def test_graph_fp64_parity_with_oracle():
    Nx, Ny, L = 64, 64, 8.0
    st = I.random_state(Nx, Ny, L, L, seed=31)
    G = O.Grid(Nx, Ny, L, L)
    phi = I.random_smooth(Nx, Ny, L, L, seed=32, kmax=4)
    vx, vy = O.dx(G, phi), O.dy(G, phi)
    z = np.zeros_like(vx)
    from paper_2306_09731_gb300.sgn import Solver
    s = Solver(Nx, Ny, L, L, graph=1, dealias=1, tol=1e-12)
    a = [dev(st.h), dev(vx), dev(vy), dev(z)]
    s.rk4_step(*a, 2e-3, 8)
    ref = O.rk4_step(G, st.h, vx, vy, z, 2e-3, 8, tol=1e-13, dealias=True)
    for x, r in zip(a[:3], ref[:3]):
        assert rel(host(x), r) < 1e-10
    s.close()


def test_graph_soliton_against_exact_solution():
    st = I.soliton_256x16()
    out, stats = run(st, 1, 100, 5e-3)
    ex = I.soliton_256x16(t=0.5)
    assert rel(out[0], ex.h) < 1e-8 and rel(out[1], ex.vx) < 1e-8
    assert stats["solves"] == 400


def test_graph_rebuilt_when_dt_changes():
    from paper_2306_09731_gb300.sgn import Solver
    st = I.random_state(64, 32, 8.0, 5.0, seed=5)
    res = []
    for graph in (1, 0):
        s = Solver(64, 32, 8.0, 5.0, graph=graph, guess=2)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        s.rk4_step(*f, 1e-3, 2)
        s.rk4_step(*f, 3e-3, 2)
        s.rk4_step(*f, 1e-3, 1)
        res.append([host(x) for x in f])
        s.close()
    for x, y in zip(*res):
        assert np.array_equal(x, y)


def test_graph_maxit_reported_and_bounded():
    """maxit stops the device-side loops exactly where the host loop stops."""
    from paper_2306_09731_gb300.sgn import Solver, SGNError, SGN_ENOTCONV
    st = I.random_state(32, 16, 6.0, 3.0, seed=4)
    res = []
    for graph in (1, 0):
        s = Solver(32, 16, 6.0, 3.0, graph=graph, tol=1e-15, maxit=3, restart=2)
        f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
        with pytest.raises(SGNError) as e:
            s.rk4_step(*f, 1e-3, 2)
        assert e.value.status == SGN_ENOTCONV
        res.append(([host(x) for x in f], s.stats()))
        s.close()
    for x, y in zip(res[0][0], res[1][0]):
        assert np.array_equal(x, y)
    assert res[0][1]["matvecs"] == res[1][1]["matvecs"] == 8 * 3
    assert res[0][1]["max_iters"] == 3


def test_graph_zero_right_hand_side():
    """v = 0: the first stage's GMRES right-hand side vanishes (sigma = 0 and
    no cycle); later stages see the flow that gravity starts."""
    st = I.random_state(64, 64, 8.0, 8.0, seed=9)
    z = np.zeros_like(st.h)
    st0 = I.State(st.Nx, st.Ny, st.Lx, st.Ly, st.h, z, z, z)
    a, sa = run(st0, 1, 2, 1e-3)
    b, sb = run(st0, 0, 2, 1e-3)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert sa["matvecs"] == sb["matvecs"] and sa["solves"] == sb["solves"] == 8


def test_graph_nonfinite_depth_reported_and_context_survives():
    from paper_2306_09731_gb300.sgn import Solver, SGNError, SGN_ENONFINITE
    st = I.random_state(32, 32, 6.0, 6.0, seed=1)
    s = Solver(32, 32, 6.0, 6.0, graph=1)
    nan = st.h.copy()
    nan[0, 0] = np.nan
    with pytest.raises(SGNError) as e:
        s.rk4_step(dev(nan), dev(st.vx), dev(st.vy), dev(st.sigma), 1e-3, 2)
    assert e.value.status == SGN_ENONFINITE
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, 1e-3, 3)
    got = [host(x) for x in f]
    s.close()
    ref, _ = run(st, 0, 3, 1e-3)
    for x, y in zip(got, ref):
        assert np.array_equal(x, y)


def test_graph_host_buffers_and_profiling_fallback():
    from paper_2306_09731_gb300.sgn import Solver, sgn_rk4_step_host
    st = I.soliton_256x16()
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, graph=1, precision=1, guess=2)
    hh = [np.ascontiguousarray(a.copy()) for a in (st.h, st.vx, st.vy, st.sigma)]
    sgn_rk4_step_host(s.handle, *hh, 5e-3, 3)
    ref, _ = run(st, 0, 3, 5e-3, precision=1, guess=2)
    for x, y in zip(hh, ref):
        assert np.array_equal(x, y)
    # profiling takes the host-driven loop: per-class times are recorded
    s.set_profiling(True)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, 5e-3, 1)
    prof = s.profile()
    assert prof["counts"]["mv_x"] > 0
    s.close()


@pytest.mark.parametrize("precision,graph,pinned", [(2, 1, True), (2, 0, True), (0, 1, True), (2, 1, False),
                                                    (0, 0, False)])
def test_host_buffer_calls_match_device_calls(precision, graph, pinned):
    """sgn_rk4_step_host copies each field on a copy stream while the others
    are transformed, from pinned or pageable arrays: the fields equal those of
    the device-buffer call bitwise, over two calls in a row, and nsteps = 0
    returns the inputs unchanged."""
    from paper_2306_09731_gb300.sgn import Solver, sgn_rk4_step_host
    st = I.perturbed_soliton(512, 64, 60.0, 15.0, a=0.5, eps=5e-2, seed=8)
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, graph=graph, precision=precision, guess=2)
    arrs = [np.ascontiguousarray(a).copy() for a in (st.h, st.vx, st.vy, st.sigma)]
    hh = [torch.tensor(a).pin_memory().numpy() for a in arrs] if pinned else arrs
    ref = [h.copy() for h in hh]
    sgn_rk4_step_host(s.handle, *hh, 2e-3, 0)
    for x, y in zip(hh, ref):
        assert np.array_equal(x, y)
    sgn_rk4_step_host(s.handle, *hh, 2e-3, 2)
    sgn_rk4_step_host(s.handle, *hh, 2e-3, 1)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s2 = Solver(st.Nx, st.Ny, st.Lx, st.Ly, graph=graph, precision=precision, guess=2)
    s2.rk4_step(*f, 2e-3, 2)
    s2.rk4_step(*f, 2e-3, 1)
    for x, y in zip(hh, f):
        assert np.array_equal(x, host(y))
    s.close()
    s2.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_extrapolation_history_across_calls(graph):
    """A call that continues the trajectory the handle returned last keeps the
    extrapolated start's history (fewer matvecs than a fresh handle on the
    same input, same fields within the FP32-bulk bar); a call on another state
    starts without it (bitwise equal to a fresh handle)."""
    from paper_2306_09731_gb300.sgn import Solver
    st = I.gaussian_hump(256, 25.0, 0.5)
    mk = lambda: Solver(256, 256, 25.0, 25.0, precision=2, guess=2, graph=graph)
    a = mk()
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    a.rk4_step(*f, 1e-3, 3)
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
    # another state: no history, the same as a fresh handle bit for bit
    pert = [x.copy() for x in mid]
    pert[0] = pert[0] + 1e-3 * np.cos(np.linspace(0.0, 2.0 * np.pi, 256))[None, :]
    p1 = [dev(x) for x in pert]
    a.rk4_step(*p1, 1e-3, 1)
    c = mk()
    p2 = [dev(x) for x in pert]
    c.rk4_step(*p2, 1e-3, 1)
    for x, y in zip(p1, p2):
        assert np.array_equal(host(x), host(y))
    for s in (a, b, c):
        s.close()
