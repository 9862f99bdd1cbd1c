"""The allocation-free elliptic operator agrees with sgn_elliptic_apply and the oracle.

sgn_elliptic_apply_noalloc serves callers that cannot allocate device memory
(an application whose own pool already holds the GPU's memory budget, a plugin
that must not allocate behind its framework's back, a loop that cannot take
cudaMalloc's implicit synchronisation). It keeps every intermediate in one
static device array shared by all calls, so each case makes two calls in a
row on different data, and the cases follow one another on different grids:
no call may see another's leftovers. The thin grids 32 x 2048, 4096 x 16 and
16 x 4096 fill the array nearly to its limit. This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import sgn_oracle as O
from paper_2306_09731_gb300 import inputs as I

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(128, 64, 10.0, 6.0, 21), (256, 256, 12.0, 12.0, 22), (32, 2048, 4.0, 120.0, 23),
         (4096, 16, 200.0, 3.0, 24), (16, 4096, 3.0, 200.0, 25)]


@pytest.mark.gpu
def test_noalloc_matches_elliptic_apply_and_oracle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09731_gb300 import sgn as S
    stream = torch.cuda.current_stream().cuda_stream
    for Nx, Ny, Lx, Ly, seed in CASES:
        G = O.Grid(Nx, Ny, Lx, Ly)
        ref_solver = S.Solver(Nx, Ny, Lx, Ly)
        for call in range(2):
            st = I.random_state(Nx, Ny, Lx, Ly, seed=seed + 100 * call)
            h, sg = _dev(st.h), _dev(st.sigma)
            out = torch.full_like(h, np.nan)
            S.sgn_elliptic_apply_noalloc(Nx, Ny, Lx, Ly, h, sg, out, stream)
            ref = ref_solver.elliptic_apply(h, sg)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.isfinite(got)), (Nx, Ny, call)
            assert _rel(got, ref.cpu().numpy()) < 1e-12, (Nx, Ny, call)
            assert _rel(got, O.elliptic_apply(G, st.h, st.sigma)) < 1e-12, (Nx, Ny, call)
        ref_solver.close()


@pytest.mark.gpu
def test_noalloc_rejects_oversized_grid():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09731_gb300 import sgn as S
    h = _dev(np.ones((512, 256)))
    out = torch.empty_like(h)
    with pytest.raises(S.SGNError) as e:
        S.sgn_elliptic_apply_noalloc(256, 512, 1.0, 1.0, h, h, out)
    assert e.value.status == S.SGN_EINVAL
    assert "65536" in str(e.value)
    with pytest.raises(S.SGNError) as e:
        S.sgn_elliptic_apply_noalloc(8192, 8, 1.0, 1.0, h, h, out)
    assert e.value.status == S.SGN_EINVAL
