"""Kernel-level parity of the CUDA path against the FP64 oracle, element by
element, on seeded inputs that span several tiles and ragged tails (empty rows,
heavy rows, beamlet counts that are not multiples of four), plus the
phantom workloads.  Tolerances are the FP32 summation bounds of tests/_helpers.
"""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import U32, need_cuda, random_case, sum_abs_cols, sum_abs_rows

pytestmark = pytest.mark.gpu


def _cases():
    yield "micro", P.make_case(P.spec_micro())
    yield "micro_ds", P.make_case(P.spec_micro(seed=21, grid=(28, 24, 10), downsample=True))
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


def _plan(case, torch, **opt):
    from paper_1003_5402_gb300 import Plan
    return Plan(case, stream=torch.cuda.current_stream().cuda_stream, **opt)


@pytest.mark.parametrize("form", ["lanes", "units", "merge"])
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_dose_spmv_and_epilogue(torch, name, case, form):
    """a1 in every form (dao_options.dose_form).  The unit and merge forms sum
    each group of 4 (FP32) or 8 entries in order and then the row's groups in
    order (a row across two warps: the two partial sums added once more): no
    term passes through more than min(n, 8) + groups <= n + 6 roundings."""
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    with _plan(case, torch, dose_form=form) as plan:
        assert plan.kernel_forms()["dose_form"] == form
        xd = torch.from_numpy(x).cuda()
        zd = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        gd = torch.empty_like(zd)
        F = plan.k_dose(xd, zd, gd)
        z = zd.cpu().numpy()
        g = gd.cpu().numpy()
    D = O.csr64(case)
    ref = O.dose(D, x.astype(np.float64))
    bound, n = sum_abs_rows(case, x)
    err = np.abs(z.astype(np.float64) - ref)
    assert np.all(err <= (n + 6) * U32 * bound + U32 * np.abs(ref)), float(np.max(err / np.maximum(bound, 1e-30)))
    vt = O.voxel_terms(case)
    # epilogue at the kernel's own z, in FP32: T - z from a hi + lo split threshold
    # (<= u), the weight rounded to FP32 and one product (<= u): |g| within 4u;
    # each F term within 4u, a lane's FP32 sum of its rows and the warp tree add
    # (rows per lane + 5) u <= 25 u for these sizes: F within 4e-6 relative
    gref = O.gradient(z.astype(np.float64), vt)
    assert np.all(np.abs(g - gref) <= 4 * U32 * np.abs(gref) + 1e-45)
    Fref = O.objective(z.astype(np.float64), vt)
    assert abs(F - Fref) <= 4e-6 * abs(Fref) + 1e-300
    Fex = O.objective(ref, vt)
    assert abs(F - Fex) <= 1e-5 * abs(Fex) + 1e-300


@pytest.mark.parametrize("dt_map,dt_threads", [("grouped", 0), ("grouped", 128), ("grouped", 256),
                                               ("consecutive", 0), ("consecutive", 128), ("consecutive", 256),
                                               ("split", 0)])
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_transposed_spmv(torch, name, case, dt_threads, dt_map):
    """a2 with a block per beamlet row (64 threads by default, or 128 or 256:
    dao_options.dt_threads) in both lane mappings, and split evenly over warps
    (dao_options.dt_map; where a row of D^T holds fewer than 32 stored entries
    the split form falls back to the consecutive one).  A thread's chain only
    gets shorter with more threads; the consecutive mapping's chain
    (ceil(n / threads) entries) is no longer than the grouped one's; a lane of
    the split form sums at most ceil(n / 32) entries, then a 5-level warp tree,
    then the warps' partials in FP64: the 64-thread grouped bound holds for all."""
    rng = np.random.default_rng(2)
    pi = rng.normal(size=case.n_voxels).astype(np.float32)
    counts = np.bincount(case.indices, minlength=case.n_beamlets)
    split_ok = int(((counts + 3) // 4 * 4).min()) >= 32
    with _plan(case, torch, dt_threads=dt_threads, dt_map=dt_map) as plan:
        assert plan.kernel_forms()["dt_map"] == (dt_map if dt_map != "split" or split_ok else "consecutive")
        pd = torch.from_numpy(pi).cuda()
        wd = torch.empty(case.n_beamlets, dtype=torch.float32, device="cuda")
        plan.k_beamlet_prices(pd, wd)
        w = wd.cpu().numpy()
    ref = O.beamlet_prices(O.csr64(case), pi.astype(np.float64))
    bound, n = sum_abs_cols(case, pi)
    err = np.abs(w.astype(np.float64) - ref)
    allowed = (np.ceil(n / 128.0) * 4 + 8) * U32 * bound + U32 * np.abs(ref)
    assert np.all(err <= allowed), float(np.max(err - allowed))


@pytest.mark.parametrize("warps", [1, 3, 100000])
@pytest.mark.parametrize("name,case", [CASES[2], CASES[3]], ids=["ragged", "heavy"])
def test_dose_merge_chunks(torch, name, case, warps):
    """The merge form of a1 with one warp (one chunk of every group), three
    warps, and a warp per chunk just longer than the longest row (most rows
    cross a boundary and are finished on its ticket; empty rows included), twice
    in a row (the tickets return to zero); z, grad F and F against the oracle."""
    rng = np.random.default_rng(6)
    x = rng.uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
    ref = O.dose(O.csr64(case), x.astype(np.float64))
    bound, n = sum_abs_rows(case, x)
    vt = O.voxel_terms(case)
    with _plan(case, torch, dose_form="merge", split_warps=warps) as plan:
        assert plan.kernel_forms()["dose_form"] == "merge"
        xd = torch.from_numpy(x).cuda()
        for _ in range(2):
            zd = torch.full((case.n_voxels,), float("nan"), dtype=torch.float32, device="cuda")
            gd = torch.full_like(zd, float("nan"))
            F = plan.k_dose(xd, zd, gd)
            z = zd.cpu().numpy().astype(np.float64)
            g = gd.cpu().numpy()
            assert np.all(np.abs(z - ref) <= (n + 6) * U32 * bound + U32 * np.abs(ref))
            gref = O.gradient(z, vt)
            assert np.all(np.abs(g - gref) <= 4 * U32 * np.abs(gref) + 1e-45)
            Fref = O.objective(z, vt)
            assert abs(F - Fref) <= 4e-6 * abs(Fref) + 1e-300


@pytest.mark.parametrize("warps", [1, 2, 7, 100000])
def test_transposed_spmv_split_chunks(torch, warps):
    """The split form of a2 with few warps (each warp's chunk spans dozens of
    rows, so its window of row offsets is refilled, and a row straddles two
    warps) and with a warp per 32 entries (every row spread over several
    warps, combined on its ticket); a second call checks that the tickets
    were left at zero."""
    case = CASES[2][1]  # ragged: rows of D^T with 44 .. ~700 entries
    rng = np.random.default_rng(5)
    pi = rng.normal(size=case.n_voxels).astype(np.float32)
    ref = O.beamlet_prices(O.csr64(case), pi.astype(np.float64))
    bound, n = sum_abs_cols(case, pi)
    allowed = (np.ceil(n / 128.0) * 4 + 8) * U32 * bound + U32 * np.abs(ref)
    with _plan(case, torch, dt_map="split", split_warps=warps) as plan:
        assert plan.kernel_forms()["dt_map"] == "split"
        pd = torch.from_numpy(pi).cuda()
        for _ in range(2):
            wd = torch.full((case.n_beamlets,), float("nan"), dtype=torch.float32, device="cuda")
            plan.k_beamlet_prices(pd, wd)
            w = wd.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(w - ref) <= allowed), float(np.nanmax(np.abs(w - ref) - allowed))


def _price_inputs(case, kind, seed):
    rng = np.random.default_rng(seed)
    N = case.n_beamlets
    if kind == "normal":
        return (rng.normal(size=N) + 0.4).astype(np.float32)
    if kind == "ties":
        return rng.integers(-3, 4, size=N).astype(np.float32)
    if kind == "positive":
        return np.abs(rng.normal(size=N)).astype(np.float32) + 1e-3
    if kind == "zeros":
        w = np.zeros(N, np.float32)
        w[rng.integers(0, N, size=max(1, N // 10))] = -1.0
        return w
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["normal", "ties", "positive", "zeros"])
@pytest.mark.parametrize("name,case", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_pricing_bit_exact_lockstep(torch, name, case, kind):
    """Fed the same FP32 w, the warp-per-row pricing equals the paper's sequential
    loop bit for bit: chosen beam, every row's [L, R), every row's v*, S_b*."""
    w = _price_inputs(case, kind, 3)
    ref = O.price(case, w.astype(np.float64))
    with _plan(case, torch) as plan:
        st, beam, leaves, rc, row_v, row_lr = plan.k_price(torch.from_numpy(w).cuda())
    assert beam == ref.beam
    assert np.array_equal(leaves, ref.leaves)
    assert rc == ref.reduced_cost
    assert np.array_equal(row_v, np.concatenate(ref.row_values))
    assert np.array_equal(row_lr, np.concatenate(ref.row_leaves))


@pytest.mark.parametrize("lanes", [0, 1, 2, 16])
@pytest.mark.parametrize("name,case", CASES, ids=[c[0] for c in CASES])
def test_aperture_column(torch, name, case, lanes):
    """a4 on D by beams (the default, dao_options.column_lanes 0: one lane per
    voxel row over the row's part of the beam, in order) and over D's row
    segments with 1, 2 or 16 lanes per row: a lane sums ceil(n / lanes)
    entries in order, then a shuffle tree of log2(lanes) levels."""
    rng = np.random.default_rng(4)
    D = O.csr64(case)
    G = lanes or 1
    with _plan(case, torch, column_lanes=lanes) as plan:
        out = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        for b in range(case.n_beams):
            R, Cn = int(case.rows[b]), int(case.cols[b])
            lv = np.zeros((R, 2), np.int32)
            for r in range(R):
                L = int(rng.integers(0, Cn + 1))
                lv[r] = (L, int(rng.integers(L, Cn + 1)))
            lv[0] = (0, Cn)                       # a full row
            if R > 1:
                lv[-1] = (0, 0)                   # a closed row
            plan.k_aperture_column(b, lv, out)
            got = out.cpu().numpy().astype(np.float64)
            ref = O.aperture_column(D, case, b, lv)
            mask = O.aperture_mask(case, b, lv)
            bound, n = sum_abs_rows(case, mask)
            assert np.all(np.abs(got - ref) <= (np.ceil(n / G) + 8) * U32 * bound + U32 * np.abs(ref)), b


def test_unit_beamlet_aperture_is_column(torch):
    """An aperture of one open beamlet gives exactly that column of D (one product
    per voxel, no rounding)."""
    case = CASES[0][1]
    D = O.csr64(case).tocsc()
    with _plan(case, torch) as plan:
        out = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        for b, r, c in [(0, 0, 0), (1, 2, 3), (case.n_beams - 1, int(case.rows[-1]) - 1, int(case.cols[-1]) - 1)]:
            lv = np.zeros((int(case.rows[b]), 2), np.int32)
            lv[r] = (c, c + 1)
            plan.k_aperture_column(b, lv, out)
            i = int(np.sum(case.rows[:b] * case.cols[:b])) + r * int(case.cols[b]) + c
            assert np.array_equal(out.cpu().numpy().astype(np.float64), D[:, i].toarray().ravel())
