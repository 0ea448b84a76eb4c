"""dao_create's device-side input checks and layout build.

Each malformed input is refused with DAO_EINVAL and the message of its first
fault: the lowest bad CSR row (its first bad entry), then the lowest bad
structure label.  The process-wide memory caches stay usable after a refused
create.  The padded row offsets come from a device scan; a matrix with more
than 4M voxel rows takes the scan of block totals through several passes, and
its stored entry count and dose must still be exact.  The transpose counts
beamlets in shared-memory tiles of 12288: a matrix with more beamlets than
one tile must give the same D^T products as the oracle.
"""
import numpy as np
import pytest

import oracle as O
from _helpers import U32, ArrayCase, need_cuda, random_case, sum_abs_cols, sum_abs_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _copy(case):
    return ArrayCase(case.indptr.copy(), case.indices.copy(), case.data.copy(), case.rows, case.cols,
                     case.voxel_struct.copy(), case.is_target, case.under_w, case.under_t, case.over_w, case.over_t)


def _refused(case, torch):
    from paper_1003_5402_gb300 import DaoError, Plan, binding
    with pytest.raises(DaoError) as e:
        Plan(case, stream=torch.cuda.current_stream().cuda_stream)
    assert e.value.status == binding.DAO_EINVAL
    return str(e.value)


def _row_with(case, min_len, start):
    ip = case.indptr
    for j in range(start, len(ip) - 1):
        if ip[j + 1] - ip[j] >= min_len:
            return j
    raise AssertionError("no such row")


BASE = random_case(41, 3001, rows=[3, 5, 2], cols=[7, 5, 13], mean_row=9.0)


def test_bad_column_nan_and_order_first_row_wins(torch):
    N = BASE.n_beamlets
    # faults planted in three rows; the lowest row's fault is reported
    c = _copy(BASE)
    j_hi = _row_with(c, 2, 2500)
    c.indices[c.indptr[j_hi]] = N                                   # column out of range
    j_mid = _row_with(c, 3, 1500)
    p = c.indptr[j_mid]
    c.indices[p], c.indices[p + 1] = c.indices[p + 1], c.indices[p]  # not increasing
    j_lo = _row_with(c, 2, 700)
    c.data[c.indptr[j_lo] + 1] = np.nan                             # non-finite value
    assert _refused(c, torch).endswith(f"non-finite value at entry {c.indptr[j_lo] + 1}")
    c.data[c.indptr[j_lo] + 1] = 0.5
    assert _refused(c, torch).endswith(f"columns not strictly increasing in row {j_mid}")
    c.indices[p], c.indices[p + 1] = c.indices[p + 1], c.indices[p]
    assert _refused(c, torch).endswith(f"column index out of range at entry {c.indptr[j_hi]}")
    c.indices[c.indptr[j_hi]] = -3
    assert _refused(c, torch).endswith(f"column index out of range at entry {c.indptr[j_hi]}")


def test_bad_row_ptr(torch):
    c = _copy(BASE)
    j = _row_with(c, 2, 1000)
    c.indptr[j + 1] = c.indptr[j] - 1                               # row j ends before it starts
    assert _refused(c, torch).endswith(f"row_ptr decreases or leaves [0, nnz] at row {j}")


def test_bad_labels_after_rows(torch):
    c = _copy(BASE)
    S = len(c.under_w)
    c.voxel_struct[2999] = S
    c.voxel_struct[1234] = -1
    assert _refused(c, torch).endswith("voxel structure label out of range at voxel 1234")
    # a CSR fault in a higher row is still reported before any label
    j = _row_with(c, 1, 2000)
    c.indices[c.indptr[j]] = 10 ** 6
    assert "column index out of range" in _refused(c, torch)


def test_valid_plan_after_refusals(torch):
    from paper_1003_5402_gb300 import Plan
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, 2.0, size=BASE.n_beamlets).astype(np.float32)
    with Plan(BASE, stream=torch.cuda.current_stream().cuda_stream) as plan:
        xd = torch.from_numpy(x).cuda()
        zd = torch.empty(BASE.n_voxels, dtype=torch.float32, device="cuda")
        plan.k_dose(xd, zd)
        z = zd.cpu().numpy().astype(np.float64)
    ref = O.dose(O.csr64(BASE), x.astype(np.float64))
    bound, n = sum_abs_rows(BASE, x)
    assert np.all(np.abs(z - ref) <= (n + 6) * U32 * bound + U32 * np.abs(ref))


def _many_rows_case(V, seed=5):
    """V voxel rows of 0..5 consecutive beamlets (one beam of 4 x 8)."""
    rng = np.random.default_rng(seed)
    L = rng.integers(0, 6, size=V).astype(np.int64)
    ip = np.zeros(V + 1, np.int64)
    np.cumsum(L, out=ip[1:])
    nnz = int(ip[-1])
    row = np.repeat(np.arange(V, dtype=np.int64), L)
    t = np.arange(nnz, dtype=np.int64) - ip[row]
    c0 = rng.integers(0, 27, size=V)
    col = (c0[row] + t).astype(np.int32)
    val = rng.uniform(0.0, 1.0, size=nnz).astype(np.float32)
    lab = rng.integers(0, 3, size=V).astype(np.int32)
    return ArrayCase(ip, col, val, [4], [8], lab, np.array([1, 0, 0], np.uint8), under_w=[10.0, 0.0, 0.0],
                     under_t=[1.0, 0.0, 0.0], over_w=[1.0, 1.0, 1.0], over_t=[1.0, 0.5, 0.5]), L


def test_row_offsets_scan_beyond_one_block_of_totals(torch):
    from paper_1003_5402_gb300 import Plan, binding
    V = 4096 * 1024 + 777                                           # > 1024 scan blocks of 4096 rows
    case, L = _many_rows_case(V)
    stream = torch.cuda.current_stream().cuda_stream
    for prec, pad in ((binding.DAO_PREC_FP32, 4), (binding.DAO_PREC_FP16, 8)):
        with Plan(case, stream=stream, precision=prec) as plan:
            assert plan.nnz_stored == int(np.sum((L + pad - 1) // pad * pad))
            if prec == binding.DAO_PREC_FP32:
                x = np.random.default_rng(9).uniform(0.0, 2.0, size=32).astype(np.float32)
                xd = torch.from_numpy(x).cuda()
                zd = torch.empty(V, dtype=torch.float32, device="cuda")
                plan.k_dose(xd, zd)
                z = zd.cpu().numpy().astype(np.float64)
    ref = O.dose(O.csr64(case), x.astype(np.float64))
    bound, n = sum_abs_rows(case, x)
    assert np.all(np.abs(z - ref) <= (n + 6) * U32 * bound + U32 * np.abs(ref))


def _tiny():
    """Six voxels, one beam of 2 x 4 beamlets (rows shorter than a warp)."""
    return ArrayCase([0, 2, 3, 3, 5, 6, 8], [0, 3, 1, 2, 7, 5, 0, 4], np.ones(8, np.float32), [2], [4],
                     [0, 0, 1, 1, 1, 1], [1, 0], under_w=[10.0, 0.0], under_t=[1.0, 0.0], over_w=[1.0, 1.0],
                     over_t=[1.0, 0.5])


@pytest.mark.parametrize("mutate,message", [
    (lambda c: c.indptr.__setitem__(2, 1), "row_ptr decreases or leaves [0, nnz] at row 1"),
    (lambda c: c.indices.__setitem__(0, 9), "column index out of range at entry 0"),
    (lambda c: c.indices.__setitem__(1, 0), "columns not strictly increasing in row 0"),
    (lambda c: c.data.__setitem__(3, np.nan), "non-finite value at entry 3"),
    (lambda c: c.voxel_struct.__setitem__(4, 7), "voxel structure label out of range at voxel 4"),
], ids=["row_ptr", "column", "order", "nan", "label"])
def test_tiny_case_faults(torch, mutate, message):
    c = _tiny()
    mutate(c)
    assert _refused(c, torch).endswith(message)


def test_transpose_with_more_beamlets_than_one_counter_tile(torch):
    from paper_1003_5402_gb300 import Plan
    case = random_case(43, 2500, rows=[300, 210], cols=[32, 31], mean_row=60.0)   # 16110 beamlets
    assert case.n_beamlets > 12288
    rng = np.random.default_rng(4)
    pi = rng.normal(size=case.n_voxels).astype(np.float32)
    with Plan(case, stream=torch.cuda.current_stream().cuda_stream) as plan:
        pd = torch.from_numpy(pi).cuda()
        wd = torch.empty(case.n_beamlets, dtype=torch.float32, device="cuda")
        plan.k_beamlet_prices(pd, wd)
        w = wd.cpu().numpy().astype(np.float64)
    ref = O.beamlet_prices(O.csr64(case), pi.astype(np.float64))
    bound, n = sum_abs_cols(case, pi)
    allowed = (np.ceil(n / 128.0) * 4 + 8) * U32 * bound + U32 * np.abs(ref)
    assert np.all(np.abs(w - ref) <= allowed)
