"""Mixed precision (16-bit values of D and D^T with a per-beamlet FP32 scale,
FP32 accumulation) against the FP64 oracle run on the dequantised matrix
s_i * RN16(D_ij / s_i), which the tests build from its definition: the same
bars as the FP32 path (FP32 summation bounds per element, leaves equal except
near-ties, objective within 1e-5).  A last test states the errors of the 16-bit
plan against the oracle on the original FP32 matrix."""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import U32, need_cuda, quantized_case, random_case, sum_abs_cols, sum_abs_rows
from test_gpu_cg import DOSE_TOL, RTOL_F, _teacher_forced

pytestmark = pytest.mark.gpu

PRECS = ["fp16", "bf16"]


def _cases():
    yield "micro", P.make_case(P.spec_micro())
    yield "ragged", random_case(31, 3001, rows=[3, 5, 2], cols=[7, 5, 13], mean_row=9.0)
    yield "heavy", random_case(32, 1203, rows=[4, 4], cols=[32, 31], mean_row=70.0)
    yield "tiny", P.make_case(P.spec_tiny())


CASES = list(_cases())


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _prec(name):
    from paper_1003_5402_gb300 import binding
    return {"fp16": binding.DAO_PREC_FP16, "bf16": binding.DAO_PREC_BF16}[name]


def _plan(case, torch, prec, **opt):
    from paper_1003_5402_gb300 import Plan
    return Plan(case, stream=torch.cuda.current_stream().cuda_stream, precision=_prec(prec), **opt)


@pytest.mark.parametrize("form", ["lanes", "units", "merge"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_dose_16bit(torch, name, case, prec, form):
    q = quantized_case(case, prec)
    x = np.random.default_rng(1).uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    with _plan(case, torch, prec, dose_form=form) as plan:
        assert plan.kernel_forms()["dose_form"] == form
        zd = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        gd = torch.empty_like(zd)
        F = plan.k_dose(torch.from_numpy(x).cuda(), zd, gd)
        z = zd.cpu().numpy().astype(np.float64)
    ref = O.dose(O.csr64(q), x.astype(np.float64))
    bound, n = sum_abs_rows(q, x)
    # the product x_i * s_i rounds once more than the FP32 path: n + 8 instead of n + 6
    assert np.all(np.abs(z - ref) <= (n + 8) * U32 * bound + U32 * np.abs(ref))
    vt = O.voxel_terms(q)
    assert abs(F - O.objective(ref, vt)) <= 1e-5 * abs(O.objective(ref, vt)) + 1e-300


@pytest.mark.parametrize("dt_map", ["grouped", "consecutive", "split"])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_transposed_16bit(torch, name, case, prec, dt_map):
    """Every form of a2; the split form where every row of D^T holds at least
    32 stored entries (rows padded to 8), else the consecutive one."""
    q = quantized_case(case, prec)
    pi = np.random.default_rng(2).normal(size=case.n_voxels).astype(np.float32)
    counts = np.bincount(case.indices, minlength=case.n_beamlets)
    split_ok = int(((counts + 7) // 8 * 8).min()) >= 32
    with _plan(case, torch, prec, dt_map=dt_map) as plan:
        assert plan.kernel_forms()["dt_map"] == (dt_map if dt_map != "split" or split_ok else "consecutive")
        wd = torch.empty(case.n_beamlets, dtype=torch.float32, device="cuda")
        plan.k_beamlet_prices(torch.from_numpy(pi).cuda(), wd)
        w = wd.cpu().numpy().astype(np.float64)
    ref = O.beamlet_prices(O.csr64(q), pi.astype(np.float64))
    bound, n = sum_abs_cols(q, pi)
    allowed = (np.ceil(n / 128.0) * 8 + 10) * U32 * bound + 2 * U32 * np.abs(ref)
    assert np.all(np.abs(w - ref) <= allowed)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_column_16bit(torch, name, case, prec):
    q = quantized_case(case, prec)
    D = O.csr64(q)
    rng = np.random.default_rng(4)
    with _plan(case, torch, prec) as plan:
        out = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        for b in range(case.n_beams):
            R, Cn = int(case.rows[b]), int(case.cols[b])
            lv = np.zeros((R, 2), np.int32)
            for r in range(R):
                L = int(rng.integers(0, Cn + 1))
                lv[r] = (L, int(rng.integers(L, Cn + 1)))
            plan.k_aperture_column(b, lv, out)
            got = out.cpu().numpy().astype(np.float64)
            ref = O.aperture_column(D, q, b, lv)
            bound, n = sum_abs_rows(q, O.aperture_mask(q, b, lv))
            assert np.all(np.abs(got - ref) <= (n / 8.0 + 8) * U32 * bound + U32 * np.abs(ref)), b


@pytest.mark.parametrize("prec", PRECS)
def test_unit_beamlet_column_is_dequantised_column(torch, prec):
    """One open beamlet: s_i * q_ij exactly (one product, exact in FP32 for
    FP16/BF16 q and FP32 s up to the product's single rounding)."""
    case = CASES[0][1]
    q = quantized_case(case, prec)
    D = O.csr64(q).tocsc()
    with _plan(case, torch, prec) as plan:
        out = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        lv = np.zeros((int(case.rows[1]), 2), np.int32)
        lv[2] = (3, 4)
        plan.k_aperture_column(1, lv, out)
        i = int(case.rows[0] * case.cols[0]) + 2 * int(case.cols[1]) + 3
        ref = D[:, i].toarray().ravel()
        got = out.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= U32 * np.abs(ref))
    assert np.array_equal(got != 0, ref != 0)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name,K", [("micro", 12), ("tiny", 16)])
def test_teacher_forced_16bit(torch, prec, name, K):
    case = P.make_case(P.CONFIGS[name]())
    q = quantized_case(case, prec)
    r = _teacher_forced(case, K, torch, plan_kw={"precision": _prec(prec)}, ref_case=q)
    Fg, Fr = np.array(r["F_gpu"]), np.array(r["F_ref"])
    assert np.all(np.abs(Fg - Fr) <= RTOL_F * np.abs(Fr)), np.abs(Fg - Fr) / np.abs(Fr)
    assert r["exact"] >= K - 2, r
    D = O.csr64(q)
    z_ref = O.dose(D, O.fluence(q, r["ref"].apertures, r["y_gpu"]))
    assert np.max(np.abs(r["z_gpu"] - z_ref)) <= DOSE_TOL
