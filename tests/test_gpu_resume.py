"""Resuming and re-planning from a saved aperture pool (dao_import_apertures).

- A pool saved from one context and imported into a fresh context on the same
  D reaches the same master optimum, and column generation continues along
  the same objective trace.
- The same pool imported on a perturbed anatomy (another D) gives the FP64
  oracle's master optimum for those apertures on that D.
- Invalid imports change nothing.
"""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import need_cuda

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _plan(case, torch, **kw):
    from paper_1003_5402_gb300 import Plan
    return Plan(case, stream=torch.cuda.current_stream().cuda_stream, **kw)


def test_import_resumes_column_generation(torch):
    case = P.make_case(P.spec_micro())
    with _plan(case, torch) as a:
        _, n, t_a = a.solve(10)
        aps, y = a.apertures(), a.intensities()
        _, _, t_more_a = a.solve(5)
    assert n == 10
    with _plan(case, torch) as b:
        F = b.import_apertures(aps, y)
        assert abs(F - t_a[9]) <= RTOL_F * abs(t_a[9]), (F, t_a[9])
        assert len(b.apertures()) == 10
        _, _, t_more_b = b.solve(5)
    assert np.all(np.abs(np.asarray(t_more_b) - np.asarray(t_more_a)) <= RTOL_F * np.abs(np.asarray(t_more_a)))


def test_import_on_another_anatomy_matches_the_oracle_master(torch):
    base = P.make_case(P.spec_micro())
    other = P.make_case(P.perturb(P.spec_micro(), 77))
    with _plan(base, torch) as a:
        a.solve(8)
        aps = a.apertures()
    with _plan(other, torch) as b:
        F = b.import_apertures(aps)
    D = O.csr64(other)
    S = np.stack([O.aperture_column(D, other, bm, lv) for bm, lv in aps], axis=1)
    ref = O.solve_master(S, O.voxel_terms(other))
    assert abs(F - ref.F) <= RTOL_F * abs(ref.F), (F, ref.F)


def test_invalid_import_changes_nothing(torch):
    from paper_1003_5402_gb300 import DaoError, binding
    case = P.make_case(P.spec_micro())
    with _plan(case, torch, k_max=4) as p:
        p.solve(2)
        before = p.apertures()
        bad = [(0, np.array([[0, 2]] * 4)), (99, np.array([[0, 1]] * 4))]
        with pytest.raises(DaoError) as e:
            p.import_apertures(bad)
        assert e.value.status == binding.DAO_EINVAL
        with pytest.raises(DaoError) as e:
            p.import_apertures([(0, np.array([[0, 1]] * 4))] * 3)  # 2 + 3 > k_max
        assert e.value.status == binding.DAO_ESTATE
        with pytest.raises(DaoError):
            p.import_apertures([(0, np.array([[0, 1]] * 4))], y_start=[-1.0])
        after = p.apertures()
    assert len(after) == len(before) == 2
    assert all(x[0] == y_[0] and np.array_equal(x[1], y_[1]) for x, y_ in zip(after, before))
