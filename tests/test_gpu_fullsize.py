"""The benchmark's workloads at full size against the FP64 oracle at every
round: 50-aperture plans on the H&N-shaped phantom (280,699 voxels, 4,500
beamlets, two nested PTVs) and the prostate-shaped phantom (161,988 voxels,
3,600 beamlets), with FP32 storage of D (oracle on the original matrix) and
FP16 storage with a per-beamlet scale (oracle on the dequantised matrix, which
the tests build from the storage's definition).

Two forms per workload and storage:
  - teacher-forced: the GPU prices from its own master optimum, the oracle's
    aperture is added on both sides (host-driven calls);
  - free-running: the device-driven graph path the benchmark times, each
    round's state read back, the oracle following the GPU's apertures.
Bars at every round: leaves equal or an accepted near-tie, objective within
1e-5 relative, dose within 1e-4 of the prescription (1.0) per voxel.  A last
test states the error of the 16-bit formats against the oracle on the original
matrix after 50 apertures.
"""
import functools

import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import need_cuda, quantized_case
from test_gpu_cg import DOSE_TOL, RTOL_F, _free_running_checked, _plan, _teacher_forced

pytestmark = pytest.mark.gpu

K = 50
FORMS = [("hn", "fp16"), ("hn", "fp32"), ("prostate", "fp32"), ("prostate", "fp16")]


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
def _ref_case(name, prec):
    c = _case(name)
    return c if prec == "fp32" else quantized_case(c, prec)


@functools.lru_cache(maxsize=None)
def _oracle(name, prec):
    """The oracle's own K-round plan of the workload and its per-round (pricing, master)."""
    steps = []
    ref = O.column_generation(_ref_case(name, prec), K, callback=lambda k, pr, m: steps.append((pr, m)))
    return ref, steps


def _kw(prec):
    from paper_1003_5402_gb300 import binding
    return {"precision": {"fp32": binding.DAO_PREC_FP32, "fp16": binding.DAO_PREC_FP16}[prec]}


@pytest.mark.parametrize("name,prec", FORMS, ids=[f"{n}-{p}" for n, p in FORMS])
def test_teacher_forced_full_size(torch, name, prec):
    r = _teacher_forced(_case(name), K, torch, plan_kw=_kw(prec), ref_case=_ref_case(name, prec),
                        ref_free=_oracle(name, prec))
    Fg, Fr = np.array(r["F_gpu"]), np.array(r["F_ref"])
    rel = np.abs(Fg - Fr) / np.abs(Fr)
    print(f"\n{name}-{prec} teacher-forced: exact {r['exact']}/{K}, ties {r['ties']}, "
          f"max objective rel {rel.max():.2e}, max dose diff {r['worst_dose']:.2e}")
    assert len(Fg) == K and np.all(rel <= RTOL_F), rel
    assert abs(r["F_dose"] - Fr[-1]) <= RTOL_F * Fr[-1]


@pytest.mark.parametrize("name,prec", FORMS, ids=[f"{n}-{p}" for n, p in FORMS])
def test_free_running_full_size(torch, name, prec):
    r = _free_running_checked(_case(name), K, torch, plan_kw=_kw(prec), ref_case=_ref_case(name, prec),
                              ref_free=_oracle(name, prec))
    print(f"\n{name}-{prec} free-running: ties {r['ties']}, max objective rel {r['worst_F_rel']:.2e}, "
          f"max dose diff {r['worst_dose']:.2e}")


def test_mixed_precision_error_statement_hn(torch):
    """The H&N-shaped workload planned with FP16 and BF16 storage, against the
    FP64 oracle on the original matrix, after 50 apertures.  Stated (printed)
    and bounded:
      - the error of the format at the plan's own fluence: the objective and
        dose the plan reports (through its stored matrix) against the same
        fluence through the original FP64 D;
      - the plan's quality: its true objective (its fluence through the
        original D) against the oracle's 50-aperture plan, one-sided, since a
        16-bit plan may take another aperture at a near-tie and end better;
      - how many leading apertures equal the oracle's.
    FP16 (11 significant bits): format error within 1e-4 of the objective and
    1e-3 of the prescription in dose, plan no worse than the oracle's by more
    than 1e-5.  BF16 (8 bits) changes the plan: 5e-2 throughout."""
    from paper_1003_5402_gb300 import binding
    case = _case("hn")
    ref, _ = _oracle("hn", "fp32")
    D = O.csr64(case)
    vt = O.voxel_terms(case)
    for prec, f_fmt, z_fmt, f_plan in (("fp16", 1e-4, 1e-3, RTOL_F), ("bf16", 5e-2, 5e-2, 5e-2)):
        pv = {"fp16": binding.DAO_PREC_FP16, "bf16": binding.DAO_PREC_BF16}[prec]
        with _plan(case, torch, precision=pv) as plan:
            st, n, trace = plan.solve(K)
            aps = plan.apertures()
            y = plan.intensities()
            z_rep, F_rep = plan.dose()
        assert n == K
        same = 0
        for k in range(n):
            if aps[k][0] == ref.apertures[k][0] and np.array_equal(aps[k][1], ref.apertures[k][1]):
                same += 1
            else:
                break
        z_true = O.dose(D, O.fluence(case, aps, y))
        F_true = O.objective(z_true, vt)
        F_ref = ref.objective[n - 1]
        fmt_F = abs(F_rep - F_true) / F_true
        fmt_z = float(np.max(np.abs(z_rep - z_true)))
        plan_F = (F_true - F_ref) / F_ref
        dz_ref = float(np.max(np.abs(z_true - ref.z)))
        print(f"\n{prec}: format error at the plan's fluence: objective {fmt_F:.3e} relative, dose {fmt_z:.3e} "
              f"(Rx 1); plan's true objective vs the oracle's {plan_F:+.3e} relative, max |dose - oracle's dose| "
              f"{dz_ref:.3e}; leading apertures equal {same}/{n}")
        assert fmt_F <= f_fmt and fmt_z <= z_fmt and plan_F <= f_plan
