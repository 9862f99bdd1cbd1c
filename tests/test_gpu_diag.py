"""sgn_diagnostics against the oracle (Sections 3, 4.1, 4.2).

Bars: the crest index, h_max, its coordinates, c_fit and max |vy| are maxima or
closed forms of the same numbers, so they match exactly. The deviations from
the solitary wave evaluate sech^2 and tanh with different libraries (the oracle
with 1/cosh^2), so they match to 1e-13 of |h| and |v|. The DFT-tail values come
from different FFTs: 1e-14 of the field's largest value (the FP64 transforms
agree to a few 1e-16 of the norm per coefficient).
"""
import math

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


def check(st, precision=0):
    from paper_2306_09731_gb300.sgn import Solver
    G = O.Grid(st.Nx, st.Ny, st.Lx, st.Ly)
    s = Solver(st.Nx, st.Ny, st.Lx, st.Ly, precision=precision)
    d = s.diagnostics(dev(st.h), dev(st.vx), dev(st.vy))
    s.close()
    r = O.diagnostics(G, st.h, st.vx, st.vy)
    for k in ("i_max", "h_max", "x_s", "y_s", "c_fit", "max_vy"):
        assert d[k] == r[k], (k, d[k], r[k])
    for k, f in (("dev_h", st.h), ("dev_vx", st.vx)):
        if math.isnan(r[k]):
            assert math.isnan(d[k])
        else:
            assert abs(d[k] - r[k]) <= 1e-13 * max(1.0, float(np.max(np.abs(f)))), (k, d[k], r[k])
    for i, f in enumerate((st.h, st.vx, st.vy)):
        assert abs(d["tail"][i] - r["tail"][i]) <= 1e-14 * max(1e-300, float(np.max(np.abs(f)))), i
    return d, r


@pytest.mark.parametrize("seed,Nx,Ny,Lx,Ly", [(1, 8, 8, 3.0, 3.0), (2, 64, 32, 8.0, 5.0), (3, 256, 16, 80.0, 10.0),
                                              (4, 32, 256, 4.0, 30.0), (5, 512, 1024, 40.0, 60.0)])
def test_diagnostics_random_states(seed, Nx, Ny, Lx, Ly):
    check(I.random_state(Nx, Ny, Lx, Ly, seed=seed))


def test_diagnostics_solitons():
    d, _ = check(I.soliton_256x16())
    assert d["dev_h"] < 1e-14 and d["max_vy"] == 0.0
    d, _ = check(I.perturbed_soliton(1024, 256, 120.0, 30.0, a=0.5, eps=5e-2, seed=7))
    assert 1e-3 < d["dev_h"] < 0.1
    check(I.deformed_soliton())


def test_diagnostics_gaussian_2048_and_precisions():
    """The benchmark workload; the diagnostics run FP64 in every precision."""
    st = I.gaussian_hump(2048, 100.0, 0.5)
    for p in (0, 2):
        check(st, precision=p)


def test_diagnostics_ties_nan_and_flat():
    st = I.random_state(32, 16, 4.0, 2.0, seed=9)
    h = np.ones((16, 32))
    h[5, 7] = 1.3
    h[2, 30] = 1.3
    check(I.State(32, 16, 4.0, 2.0, h, st.vx, st.vy, st.sigma))
    check(I.State(32, 16, 4.0, 2.0, np.ones((16, 32)), st.vx, st.vy, st.sigma))
    hn = st.h.copy()
    hn[4, 3] = np.nan
    hn[9, 1] = np.nan
    from paper_2306_09731_gb300.sgn import Solver
    s = Solver(32, 16, 4.0, 2.0)
    d = s.diagnostics(dev(hn), dev(st.vx), dev(st.vy))
    s.close()
    assert math.isnan(d["h_max"]) and d["i_max"] == 4 * 32 + 3 == int(np.argmax(hn))
