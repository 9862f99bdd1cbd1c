"""Ensembles: sgn_rk4_step_batch over uneven grids.

Each member is exactly the single-member computation on its own handle and
stream, so the bar is bitwise equality with sgn_rk4_step member by member, and
one member's failure must not touch the others.
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


GRIDS = [(64, 64, 30.0, 30.0), (128, 64, 60.0, 30.0), (256, 128, 60.0, 30.0)]


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("graph", [1, 0])
def test_batch_equals_members_one_by_one(graph):
    from paper_2306_09731_gb300.ensemble import Ensemble, perturbed_members
    states = perturbed_members(7, seed=3, grids=GRIDS)
    a = Ensemble(states, precision=2, guess=2, graph=graph)
    st = a.step(2e-3, 4)
    assert st == [0] * 7
    b = Ensemble(states, precision=2, guess=2, graph=graph)
    b.step_one_by_one(2e-3, 4)
    for fa, fb in zip(a.fields, b.fields):
        for x, y in zip(fa, fb):
            assert np.array_equal(host(x), host(y))
    for sa, sb in zip(a.solvers, b.solvers):
        assert sa.stats()["matvecs"] == sb.stats()["matvecs"]
    a.close()
    b.close()


def test_failing_member_is_isolated():
    from paper_2306_09731_gb300.ensemble import Ensemble, perturbed_members
    from paper_2306_09731_gb300.sgn import SGNError, SGN_ENONFINITE
    states = perturbed_members(4, seed=5, grids=GRIDS)
    bad = states[2]
    bad.h = bad.h.copy()
    bad.h[3, 4] = np.nan
    e = Ensemble(states, precision=2, guess=2, graph=1)
    with pytest.raises(SGNError) as err:
        e.step(2e-3, 2)
    assert err.value.status == SGN_ENONFINITE
    ok = Ensemble([states[i] for i in (0, 1, 3)], precision=2, guess=2, graph=1)
    ok.step_one_by_one(2e-3, 2)
    for i, j in ((0, 0), (1, 1), (3, 2)):
        for x, y in zip(e.fields[i], ok.fields[j]):
            assert np.array_equal(host(x), host(y))
    e.close()
    ok.close()
