"""The allocation-free elliptic operator agrees with sgn_elliptic_apply.

sgn_elliptic_apply_noalloc serves callers that cannot allocate device memory
(an application whose own pool already holds the GPU's memory budget, a plugin
that must not allocate behind its framework's back, a loop that cannot take
cudaMalloc's implicit synchronisation). It keeps every intermediate in one
static device array shared by all calls, so this test makes two calls in a
row on different grids and data: the second must not see the first's leftovers.
This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

from paper_2306_09731_gb300 import inputs as I

torch = pytest.importorskip("torch")


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
def test_noalloc_matches_elliptic_apply_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2306_09731_gb300 import sgn as S
    cases = [(128, 64, 10.0, 6.0, 21), (256, 256, 12.0, 12.0, 22)]
    for Nx, Ny, Lx, Ly, seed in cases:
        st = I.random_state(Nx, Ny, Lx, Ly, seed=seed)
        h, sg = _dev(st.h), _dev(st.sigma)
        stream = torch.cuda.current_stream().cuda_stream
        out = torch.full_like(h, np.nan)
        S.sgn_elliptic_apply_noalloc(Nx, Ny, Lx, Ly, h, sg, out, stream)
        ref_solver = S.Solver(Nx, Ny, Lx, Ly)
        ref = ref_solver.elliptic_apply(h, sg)
        torch.cuda.synchronize()
        ref_solver.close()
        assert _rel(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12


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
