"""Beamlet-level FMO on the GPU (dao_fmo; Sec. 2.2-2.3: min over x >= 0 of
F(D x), the DAO model with beamlets as the decision variables) against the
FP64 oracle's FMO (projected Newton with exact factorisations, itself pinned
against L-BFGS-B): the objective within 1e-5 relative of the oracle's optimum,
the GPU's x a KKT point of the FP64 problem, and the FMO optimum a lower bound
of the GPU's own DAO plans."""
import functools

import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import need_cuda, quantized_case
from test_gpu_cg import _plan

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


@functools.lru_cache(maxsize=None)
def _case(name):
    return P.make_case(P.CONFIGS[name]())


def _golden_fmo():
    """Stored oracle optima of the full-size workloads (tests/golden/make_fmo_optima.py)."""
    import os
    out = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fmo_optima.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            out[f[0]] = float(f[1])
    return out


def _kkt_rel(case, x, vt=None):
    """max over beamlets of |min(x_i, g_i)| / max|g(0)| in FP64: 0 at the optimum."""
    D = O.csr64(case)
    vt = O.voxel_terms(case) if vt is None else vt
    g = D.T @ O.gradient(D @ x, vt)
    g0 = D.T @ O.gradient(np.zeros(case.n_voxels), vt)
    return float(np.max(np.abs(np.minimum(x, g)))) / float(np.max(np.abs(g0)))


@pytest.mark.parametrize("name,prec", [("micro", 0), ("tiny", 0), ("tiny", 1), ("prostate", 0)],
                         ids=["micro", "tiny", "tiny-fp16", "prostate"])
def test_fmo_matches_oracle(torch, name, prec):
    case = _case(name)
    ref_case = case if prec == 0 else quantized_case(case, "fp16")
    gold = _golden_fmo()
    ref_F = gold[name] if (prec == 0 and name in gold) else O.fmo(ref_case).F
    with _plan(case, torch, precision=prec) as plan:
        st, x, F, its, cg = plan.fmo(max_iters=300, tol=1e-7)
    print(f"\nFMO {name} prec={prec}: F {F:.9e} oracle {ref_F:.9e} rel {(F - ref_F) / ref_F:+.2e}, "
          f"{its} Newton steps, {cg} CG iterations, status {st}")
    assert np.all(x >= 0)
    assert abs(F - ref_F) <= RTOL_F * ref_F
    assert _kkt_rel(ref_case, x) <= 1e-4


def test_fmo_bounds_the_dao_plans(torch):
    case = _case("tiny")
    with _plan(case, torch) as plan:
        _, x, F_fmo, _, _ = plan.fmo()
        st, n, trace = plan.solve(30)
    assert np.all(trace[:n] >= F_fmo * (1 - 1e-6))
    # the pool is untouched by dao_fmo: the DAO plan is the oracle's
    ref = O.column_generation(case, 5)
    assert np.all(np.abs(trace[:5] - ref.objective) <= RTOL_F * np.array(ref.objective))


def test_fmo_reoptimisation_mode(torch):
    """FMO on per-voxel terms (the re-optimisation form of Eqs. 3-4)."""
    case = _case("micro")
    z0 = O.column_generation(case, 4).z
    xyz = np.asarray(case.voxel_xyz, np.float64)
    T = z0 * (1.0 + 0.05 * np.sin(2 * np.pi * xyz[:, 0] / 20.0))   # a smoothly deformed planned dose
    vt = O.reoptimisation_terms(T, target_mask=np.asarray(case.is_target, bool)[case.voxel_struct])
    ref = O.fmo(case, vt=vt)
    with _plan(case, torch, voxel_terms=(vt.alpha, vt.t_under, vt.beta, vt.t_over)) as plan:
        st, x, F, its, cg = plan.fmo(max_iters=300, tol=1e-7)
    assert ref.F > 1e-8 and abs(F - ref.F) <= RTOL_F * ref.F
    assert _kkt_rel(case, x, vt) <= 1e-4


def test_fmo_argument_checks(torch):
    from paper_1003_5402_gb300 import DaoError
    with _plan(_case("micro"), torch) as plan:
        with pytest.raises(DaoError):
            plan.fmo(max_iters=0)
        with pytest.raises(DaoError):
            plan.fmo(tol=0.0)
