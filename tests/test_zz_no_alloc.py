"""The allocation-free dose entry point (dao_dose_objective_noalloc).

It serves callers that must not allocate device memory while they run: a
re-planning service that reserves every device buffer before an online adaptive
fraction, so the fraction cannot fail on an allocation or stall on the
synchronisation that cudaMalloc / cudaFree may imply, or an application whose
own allocator owns the device.  Its scratch memory is a file-scope device array
shared by every call, so two calls in a row must both match the context-based
dao_k_dose, and a problem above the array's limit must be refused.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import phantom as P
from _helpers import U32, need_cuda, sum_abs_rows

pytestmark = pytest.mark.gpu


def _terms(case):
    """Per-structure (alpha_s/|v_s|, T_s^-, beta_s/|v_s|, T_s^+) as the context builds them."""
    S = len(case.under_w)
    count = np.bincount(np.asarray(case.voxel_struct), minlength=S).astype(np.float64)
    vol = np.where(count > 0, count, 1.0)
    tgt = np.asarray(case.is_target).astype(bool)
    out = np.zeros((S, 4))
    out[:, 0] = np.where(tgt, case.under_w / vol, 0.0)
    out[:, 1] = np.where(tgt, case.under_t, 0.0)
    out[:, 2] = case.over_w / vol
    out[:, 3] = case.over_t
    return out


@pytest.mark.parametrize("name", ["micro", "tiny"])
def test_noalloc_dose_matches_context_dose_on_two_calls(name):
    torch = need_cuda()
    from paper_1003_5402_gb300 import Plan, binding, build
    build.build()
    case = P.make_case(P.CONFIGS[name]())
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(17)
    x_h = rng.uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    x = torch.from_numpy(x_h).cuda()
    with Plan(case, stream=stream.cuda_stream) as plan:
        z_ref = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        g_ref = torch.empty_like(z_ref)
        F_ref = plan.k_dose(x, z_ref, g_ref)
    z_ref, g_ref = z_ref.cpu().numpy(), g_ref.cpu().numpy()

    row_ptr = torch.from_numpy(case.indptr.astype(np.int32)).cuda()
    col = torch.from_numpy(case.indices).cuda()
    val = torch.from_numpy(case.data).cuda()
    vs = torch.from_numpy(case.voxel_struct.astype(np.int32)).cuda()
    terms = _terms(case)
    bound, n = sum_abs_rows(case, x_h)
    z_tol = 2 * (n + 6) * U32 * bound + 2 * U32 * np.abs(z_ref)
    ab = np.abs(terms[case.voxel_struct, 0]) + np.abs(terms[case.voxel_struct, 2])
    for call in range(2):
        z = torch.full((case.n_voxels,), float("nan"), dtype=torch.float32, device="cuda")
        g = torch.full_like(z, float("nan"))
        F = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        binding.dose_objective_noalloc(row_ptr, col, val, x, vs, terms, z, g, F, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        zn, gn, Fn = z.cpu().numpy(), g.cpu().numpy(), float(F.item())
        assert np.all(np.abs(zn - z_ref) <= z_tol), (call, float(np.max(np.abs(zn - z_ref) - z_tol)))
        assert np.all(np.abs(gn - g_ref) <= 2 * ab * z_tol + 4 * U32 * np.abs(g_ref) + 1e-30), call
        assert abs(Fn - F_ref) <= 1e-5 * abs(F_ref), (call, Fn, F_ref)


def test_noalloc_refuses_problems_above_its_scratch_limit():
    torch = need_cuda()
    from paper_1003_5402_gb300 import binding, build
    build.build()
    lib = binding.load()
    small_i = torch.zeros(8, dtype=torch.int32, device="cuda")
    small_f = torch.zeros(8, dtype=torch.float32, device="cuda")
    out_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    terms = np.zeros((1, 4))
    P_ = lambda t: C.c_void_p(t.data_ptr())
    st = lib.dao_dose_objective_noalloc(4_194_305, 8, P_(small_i), P_(small_i), P_(small_f), P_(small_f), P_(small_i),
                                        1, terms.ctypes.data_as(C.POINTER(C.c_double)), P_(small_f), None, P_(out_d),
                                        None)
    assert st == binding.DAO_EINVAL
    assert "4194304" in lib.dao_last_error().decode()


def _micro_inputs(torch):
    case = P.make_case(P.spec_micro())
    rng = np.random.default_rng(23)
    x_h = rng.uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    return (case, x_h, dev(case.indptr, np.int32), dev(case.indices, np.int32), dev(case.data, np.float32),
            dev(x_h, np.float32), dev(case.voxel_struct, np.int32))


def test_noalloc_without_gradient_matches_context_dose():
    """grad = NULL: only z and the objective, still equal to dao_k_dose's."""
    torch = need_cuda()
    from paper_1003_5402_gb300 import Plan, binding, build
    build.build()
    case, x_h, row_ptr, col, val, x, vs = _micro_inputs(torch)
    stream = torch.cuda.current_stream()
    with Plan(case, stream=stream.cuda_stream) as plan:
        z_ref = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        F_ref = plan.k_dose(x, z_ref, None)
    z_ref = z_ref.cpu().numpy()
    bound, n = sum_abs_rows(case, x_h)
    z_tol = 2 * (n + 6) * U32 * bound + 2 * U32 * np.abs(z_ref)
    for call in range(2):
        z = torch.full((case.n_voxels,), float("nan"), dtype=torch.float32, device="cuda")
        F = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        binding.dose_objective_noalloc(row_ptr, col, val, x, vs, _terms(case), z, None, F, stream=stream)
        torch.cuda.synchronize()
        assert np.all(np.abs(z.cpu().numpy() - z_ref) <= z_tol), call
        assert abs(float(F.item()) - F_ref) <= 1e-5 * abs(F_ref), (call, float(F.item()), F_ref)


def test_noalloc_flags_a_label_out_of_range():
    """A label outside [0, n_structures) is never used as an index: that voxel's
    derivative and the objective come back NaN, the dose is still written, and
    the next call with valid labels is exact again."""
    torch = need_cuda()
    from paper_1003_5402_gb300 import binding, build
    build.build()
    case, x_h, row_ptr, col, val, x, vs = _micro_inputs(torch)
    terms = _terms(case)
    bad = vs.clone()
    bad[5] = 64
    bad[9] = -1
    z = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
    g = torch.empty_like(z)
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    binding.dose_objective_noalloc(row_ptr, col, val, x, bad, terms, z, g, F)
    torch.cuda.synchronize()
    gn = g.cpu().numpy()
    assert np.isnan(float(F.item()))
    assert np.isnan(gn[5]) and np.isnan(gn[9]) and np.count_nonzero(np.isnan(gn)) == 2
    assert np.all(np.isfinite(z.cpu().numpy()))
    binding.dose_objective_noalloc(row_ptr, col, val, x, vs, terms, z, g, F)
    torch.cuda.synchronize()
    assert np.isfinite(float(F.item())) and np.all(np.isfinite(g.cpu().numpy()))


def test_noalloc_runs_on_the_tensors_device_and_refuses_a_foreign_stream():
    """With another device current, the wrapper still runs on the tensors'
    device; a stream of another device is refused by the library."""
    torch = need_cuda()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    from paper_1003_5402_gb300 import DaoError, binding, build
    build.build()
    case, x_h, row_ptr, col, val, x, vs = _micro_inputs(torch)   # on cuda:0
    z = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda:0")
    F = torch.empty(1, dtype=torch.float64, device="cuda:0")
    with torch.cuda.device(1):
        binding.dose_objective_noalloc(row_ptr, col, val, x, vs, _terms(case), z, None, F)
    torch.cuda.synchronize(0)
    assert np.isfinite(float(F.item()))
    other = torch.cuda.Stream(device=1)
    with pytest.raises(ValueError):
        binding.dose_objective_noalloc(row_ptr, col, val, x, vs, _terms(case), z, None, F, stream=other)
    with pytest.raises(DaoError):
        binding.dose_objective_noalloc(row_ptr, col, val, x, vs, _terms(case), z, None, F,
                                       stream=other.cuda_stream)
