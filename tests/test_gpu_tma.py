"""Tensor-copied inputs of the FP32 matvec y-passes (precisions 1 and 2).

The tiles that the tensor engine copies hold the same values that the plain
loads read, and the transforms and epilogues are the same code, so the bar is
bitwise equality with the handle made under SGN_TMA=0 (plain loads), on the
shapes whose tiles differ: 2 to 64 columns per block, ragged last tiles
(Nx/2 + 1 is odd), box heights below 256 rows, and 4096-point columns.
"""
import os

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


def run(st, tma, steps, dt, **opts):
    from paper_2306_09731_gb300.sgn import Solver
    old = os.environ.get("SGN_TMA")
    os.environ["SGN_TMA"] = "1" if tma else "0"
    try:
        s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, **opts)
    finally:
        if old is None:
            del os.environ["SGN_TMA"]
        else:
            os.environ["SGN_TMA"] = old
    f = [dev(st.h), dev(st.vx), dev(st.vy), dev(st.sigma)]
    s.rk4_step(*f, dt, steps)
    torch.cuda.synchronize()
    out = [x.cpu().numpy() for x in f]
    stats = s.stats()
    s.close()
    return out, stats


@pytest.mark.parametrize("Nx,Ny,Lx,Ly", [(8, 8, 3.0, 3.0), (64, 16, 8.0, 3.0), (256, 64, 60.0, 15.0),
                                         (2048, 8, 100.0, 2.0), (16, 2048, 3.0, 100.0), (4096, 16, 200.0, 4.0)])
@pytest.mark.parametrize("precision,graph", [(1, 0), (2, 1)])
def test_tma_inputs_bitwise_equal_to_plain_loads(Nx, Ny, Lx, Ly, precision, graph):
    st = I.random_band_state(Nx, Ny, Lx, Ly, seed=Nx + 3 * Ny, kx_max=min(20, Nx // 4), ky_max=min(6, Ny // 4))
    a, sa = run(st, True, 4, 1e-3, precision=precision, graph=graph, guess=2)
    b, sb = run(st, False, 4, 1e-3, precision=precision, graph=graph, guess=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert sa["matvecs"] == sb["matvecs"] and sa["solves"] == sb["solves"] == 16


def test_tma_benchmark_state_bitwise():
    """The 2048^2 benchmark state, two steps of the headline path."""
    st = I.gaussian_hump(2048, 100.0, 0.5)
    a, sa = run(st, True, 2, 1e-3, precision=2, graph=1, guess=2)
    b, sb = run(st, False, 2, 1e-3, precision=2, graph=1, guess=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert sa["matvecs"] == sb["matvecs"]
