"""sgn_autotune: launch shapes and radix plans of the transform passes picked by timing.

A shape only changes how columns (row pairs) are grouped into blocks. The
FP64 passes run the same kernels in every shape: bitwise equality of the
fields and GMRES statistics with an untuned handle when the tuner kept radix
plan 0 everywhere; a pass whose radix-2/4 stage moved first (plan 1) rounds
differently, so with any plan 1 picked the FP64 fields agree to 1e-12 and
every solve still meets the tolerance. An FP32 pass in a shape
other than the built-in one runs the kernel compiled for runtime lengths,
which may fuse multiply-adds differently (last-bit differences in the inner
solve and the FP32 RHS); every solve still meets the FP64 tolerance, so the
fields agree to 1e-6 relative (the FP32 rounding of one RHS, ~1e-7, times the
few steps), with the same number of solves. Grids: those whose built-in shapes
leave few blocks (256^2 and the ensemble grids), thin grids, 4096-point axes.
"""
import numpy as np
import pytest

from paper_2306_09731_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def cuda_ready():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def run(st, tune, steps, **opts):
    from paper_2306_09731_gb300.sgn import Solver
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, **opts)
    tuning = s.autotune(3) if tune else None
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, 1e-3, steps)
    torch.cuda.synchronize()
    out = [x.cpu().numpy() for x in f]
    stats = s.stats()
    s.close()
    return out, stats, tuning


GRIDS = [(256, 256, 30.0, 30.0), (512, 256, 60.0, 30.0), (1024, 512, 120.0, 60.0), (64, 16, 8.0, 3.0),
         (2048, 64, 100.0, 5.0), (4096, 16, 200.0, 4.0)]


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", GRIDS)
@pytest.mark.parametrize("precision,graph", [(0, 0), (2, 1)])
def test_tuned_shapes_bitwise_equal(Nx, Ny, Lx, Ly, precision, graph):
    st = I.random_band_state(Nx, Ny, Lx, Ly, seed=Nx + Ny, kx_max=min(20, Nx // 4), ky_max=min(6, Ny // 4))
    a, sa, tuning = run(st, True, 3, precision=precision, graph=graph, guess=2)
    b, sb, _ = run(st, False, 3, precision=precision, graph=graph, guess=2)
    plans = [r["plan"] for passes in tuning.values() for r in passes.values()]
    if precision == 0 and not any(plans):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        assert sa["matvecs"] == sb["matvecs"]
    elif precision == 0:
        for x, y in zip(a, b):
            assert np.linalg.norm(x - y) <= 1e-12 * max(np.linalg.norm(y), 1e-300)
    else:
        for x, y in zip(a, b):
            assert np.linalg.norm(x - y) <= 1e-6 * max(np.linalg.norm(y), 1e-300)
    assert sa["solves"] == sb["solves"]
    # every pass the precision runs was timed; the pick is the fastest shape,
    # the built-in one included
    types = {"fp64"} if precision == 0 else {"fp32", "dfl"}
    assert set(tuning) == types
    for ty, passes in tuning.items():
        for ps, r in passes.items():
            assert r["us"] <= r["us_default"]
            assert r["threads"] % 32 == 0 or r["threads"] == r["default_threads"]
            # one plan when 3 divides log2 of the pass's axis length
            n = Nx if ps.endswith("_x") else Ny
            assert r["plan"] in (0, 1) and (r["plan"] == 0 or int(np.log2(n)) % 3 != 0)


def test_autotune_rejects_bad_reps_and_retunes():
    from paper_2306_09731_gb300.sgn import SGNError, SGN_EINVAL, Solver
    s = Solver(64, 64, 8.0, 8.0, precision=1)
    with pytest.raises(SGNError) as e:
        s.autotune(0)
    assert e.value.status == SGN_EINVAL
    t1 = s.autotune(2)
    t2 = s.autotune(2)
    assert set(t1) == set(t2) == {"fp32", "fp64"}
    s.close()


# axes of every residue of log2 N mod 3: 1024 (plan 1 has a radix-2 stage
# first), 2048 and 32 (radix-4 first), 64 and 512 (one plan)
PLAN_GRIDS = [(1024, 32, 100.0, 6.0), (64, 2048, 8.0, 100.0), (512, 512, 40.0, 40.0)]


def all_plan1(tuning):
    return {ty: {ps: {"threads": 0, "plan": 1} for ps in passes} for ty, passes in tuning.items()}


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", PLAN_GRIDS)
@pytest.mark.parametrize("precision,bar", [(0, 1e-10), (2, 1e-5)])
def test_radix_plan1_against_oracle(Nx, Ny, Lx, Ly, precision, bar):
    """Every pass forced to radix plan 1 (sgn_set_tuning): one RHS and two RK4
    steps against the oracle at the precision's bar (Section 3)."""
    from oracle import sgn_oracle as O
    from paper_2306_09731_gb300.sgn import Solver
    st = I.random_band_state(Nx, Ny, Lx, Ly, seed=3 * Nx + Ny, kx_max=min(30, Nx // 4), ky_max=min(30, Ny // 4))
    G = O.Grid(Nx, Ny, Lx, Ly)
    s = Solver(Nx, Ny, Lx, Ly, precision=precision, tol=1e-12, guess=2, graph=1)
    s.set_tuning(all_plan1(s.autotune(1)))
    sg = dev(st.sigma)
    ht, vxt, vyt = s.rhs(dev(st.h), dev(st.vx), dev(st.vy), sg)
    ref = O.rhs(G, st.h, st.vx, st.vy, st.sigma, tol=1e-13)
    for a, r in zip((ht, vxt, vyt), ref[:3]):
        torch.cuda.synchronize()
        assert np.linalg.norm(a.cpu().numpy() - r) <= bar * np.linalg.norm(r)
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, 1e-3, 2)
    ref = O.rk4_step(G, st.h, st.vx, st.vy, st.sigma, 1e-3, 2, tol=1e-13)
    for a, r in zip(f[:3], ref[:3]):
        torch.cuda.synchronize()
        assert np.linalg.norm(a.cpu().numpy() - r) <= bar * np.linalg.norm(r)
    s.close()


def test_set_tuning_rejects_bad_shapes_and_plans():
    from paper_2306_09731_gb300.sgn import SGNError, SGN_EINVAL, Solver
    s = Solver(256, 256, 30.0, 30.0, precision=2)
    t = s.autotune(1)
    bad = {ty: {ps: dict(r, plan=2) for ps, r in passes.items()} for ty, passes in t.items()}
    with pytest.raises(SGNError) as e:
        s.set_tuning(bad)
    assert e.value.status == SGN_EINVAL
    bad = {"fp32": {"mv_x": {"threads": 96, "plan": 0}}}
    with pytest.raises(SGNError) as e:
        s.set_tuning(bad)
    assert e.value.status == SGN_EINVAL
    s.set_tuning(t)  # a tuning the tuner returned applies as is
    s.close()
