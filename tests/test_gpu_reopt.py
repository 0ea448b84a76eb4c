"""Re-optimisation mode on the GPU (Sec. 4: Eqs. 3-4 with alpha_j = beta_j = 1
and T_j the planned dose deformed onto the day's anatomy) against the FP64
oracle given the same per-voxel terms.

Input recipe: the planned dose z0 is the oracle's own plan of the case (a few
apertures); the "deformation" is a shift of one voxel (2.5 mm) along x on the
regular grid of the small box (voxels without a source voxel get 0), or, on the
down-sampled prostate-shaped grid, a smooth seeded multiplicative field of
+-5 %.  Eq. 3 applies to target voxels, Eq. 4 to all voxels.  The bars are
those of the structure-based plans: leaves equal or an accepted near-tie,
objective within 1e-5, dose within 1e-4 per voxel at every round.
"""
import functools

import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import U32, need_cuda, sum_abs_rows
from test_gpu_cg import RTOL_F, _free_running_checked, _plan, _teacher_forced

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


@functools.lru_cache(maxsize=None)
def _case(name):
    return P.make_case(P.CONFIGS[name]())


@functools.lru_cache(maxsize=None)
def _reopt(name, k_plan=6):
    """(oracle terms, plan kwargs) of the re-optimisation workload on ``name``."""
    case = _case(name)
    z0 = O.column_generation(case, k_plan).z
    xyz = np.asarray(case.voxel_xyz, np.float64)
    if name == "prostate":
        u = P.uniform(77, np.arange(2))
        f = 1.0 + 0.05 * np.sin(2 * np.pi * (xyz[:, 0] / 80.0 + u[0])) * np.cos(2 * np.pi * (xyz[:, 1] / 60.0 + u[1]))
        T = z0 * f
    else:
        h = case.spec.voxel_mm
        key = {tuple(np.round(p / h * 2).astype(np.int64)): j for j, p in enumerate(xyz)}
        src = [key.get(tuple(np.round((p - (h, 0.0, 0.0)) / h * 2).astype(np.int64)), -1) for p in xyz]
        src = np.array(src)
        T = np.where(src >= 0, z0[np.maximum(src, 0)], 0.0)
    tgt = np.asarray(case.is_target, bool)[np.asarray(case.voxel_struct)]
    vt = O.reoptimisation_terms(T, target_mask=tgt)
    terms = (vt.alpha, vt.t_under, vt.beta, vt.t_over)
    return vt, terms


@pytest.mark.parametrize("name", ["micro", "tiny"])
def test_reopt_dose_epilogue(torch, name):
    case = _case(name)
    vt, terms = _reopt(name)
    x = np.random.default_rng(5).uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    with _plan(case, torch, voxel_terms=terms) as plan:
        zd = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        gd = torch.empty_like(zd)
        F = plan.k_dose(torch.from_numpy(x).cuda(), zd, gd)
        z, g = zd.cpu().numpy(), gd.cpu().numpy()
    ref = O.dose(O.csr64(case), x.astype(np.float64))
    bound, n = sum_abs_rows(case, x)
    assert np.all(np.abs(z - ref) <= (n + 6) * U32 * bound + U32 * np.abs(ref))
    gref = O.gradient(z.astype(np.float64), vt)
    assert np.all(np.abs(g - gref) <= 4 * U32 * np.abs(gref) + 1e-45)
    Fref = O.objective(z.astype(np.float64), vt)
    assert abs(F - Fref) <= 4e-6 * abs(Fref)


@pytest.mark.parametrize("persistent", [1, 0])
@pytest.mark.parametrize("name,K", [("micro", 12), ("tiny", 20)])
def test_reopt_teacher_forced(torch, name, K, persistent):
    case = _case(name)
    vt, terms = _reopt(name)
    r = _teacher_forced(case, K, torch, plan_kw={"voxel_terms": terms, "master_persistent": persistent}, vt=vt)
    Fg, Fr = np.array(r["F_gpu"]), np.array(r["F_ref"])
    assert np.all(np.abs(Fg - Fr) <= RTOL_F * np.abs(Fr)), np.abs(Fg - Fr) / np.abs(Fr)
    assert r["exact"] >= K - 2, r
    assert abs(r["F_dose"] - Fr[-1]) <= RTOL_F * Fr[-1]


@pytest.mark.parametrize("name,K,prec", [("tiny", 20, 0), ("prostate", 30, 0), ("prostate", 30, 1)],
                         ids=["tiny-fp32", "prostate-fp32", "prostate-fp16"])
def test_reopt_free_running(torch, name, K, prec):
    """The device-driven graph path in re-optimisation mode, every round against
    the oracle (16-bit storage against the dequantised matrix)."""
    from _helpers import quantized_case
    case = _case(name)
    vt, terms = _reopt(name)
    ref_case = case if prec == 0 else quantized_case(case, "fp16")
    r = _free_running_checked(case, K, torch, plan_kw={"voxel_terms": terms, "precision": prec},
                              ref_case=ref_case, vt=vt)
    print(f"\nre-optimisation {name} prec={prec}: ties {r['ties']}, max objective rel {r['worst_F_rel']:.2e}, "
          f"max dose diff {r['worst_dose']:.2e}")


def test_reopt_graph_rounds_equal_host_driven(torch):
    case = _case("micro")
    vt, terms = _reopt("micro")
    out = []
    for g in (1, 0):
        with _plan(case, torch, voxel_terms=terms, use_graphs=g) as plan:
            st, n, trace = plan.solve(16)
            out.append((n, trace, plan.apertures(), plan.intensities(), plan.dose()))
    a, b = out
    assert a[0] == b[0] and np.array_equal(a[1], b[1], equal_nan=True) and np.array_equal(a[3], b[3])
    assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(a[2], b[2]))
    assert np.array_equal(a[4][0], b[4][0]) and a[4][1] == b[4][1]


def test_reopt_rejects_invalid_terms(torch):
    from paper_1003_5402_gb300 import DaoError
    case = _case("micro")
    V = case.n_voxels
    ok = [np.ones(V), np.ones(V), np.ones(V), np.ones(V)]
    for k, bad in ((0, -1.0), (2, np.inf), (1, np.nan), (3, np.inf)):
        t = [a.copy() for a in ok]
        t[k][V // 2] = bad
        with pytest.raises(DaoError) as e:
            _plan(case, torch, voxel_terms=t)
        assert e.value.status == -1
    with pytest.raises(ValueError):
        _plan(case, torch, voxel_terms=[np.ones(V)] * 3)
