"""Batched plans (dao_batch_solve) and the SpMV autotuner (dao_autotune).

A batch runs every instance's rounds as its own CUDA graphs on its own stream;
the instances share no device state, so each one's apertures, intensities,
objective trace and dose must equal, bit for bit, those of the same instance
solved alone.  The autotuner's choice must come from its candidate sets, be
read back from its cache for the same size class, and leave the kernels within
the FP32 parity bounds against the oracle."""
import numpy as np
import pytest

import oracle as O
import phantom as P
from _helpers import U32, need_cuda, random_case, sum_abs_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _instances():
    micro = P.spec_micro()
    return [
        ("micro", P.make_case(micro), {}),
        ("micro@4001", P.make_case(P.perturb(micro, 4001)), {}),
        ("micro@4002", P.make_case(P.perturb(micro, 4002)), {}),
        ("tiny", P.make_case(P.spec_tiny()), {}),
        ("ragged", random_case(31, 3001, rows=[3, 5, 2], cols=[7, 5, 13], mean_row=9.0), {}),
        ("micro_fp16", P.make_case(micro), {"precision": 1}),
    ]


def _snapshot(plan, res):
    st, n, trace = res
    z, F = plan.dose()
    return st, n, trace, plan.apertures(), plan.intensities(), z, F


def _same(a, b):
    assert a[0] == b[0] and a[1] == b[1]
    assert np.array_equal(a[2], b[2], equal_nan=True)
    assert len(a[3]) == len(b[3])
    assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(a[3], b[3]))
    assert np.array_equal(a[4], b[4]) and np.array_equal(a[5], b[5]) and a[6] == b[6]


def test_batch_equals_each_instance_alone_bitwise(torch):
    from paper_1003_5402_gb300 import Plan, binding
    K = 12
    inst = _instances()
    alone = []
    for name, case, kw in inst:
        with Plan(case, **kw) as p:
            alone.append(_snapshot(p, p.solve(K)))
    plans = [Plan(case, **kw) for name, case, kw in inst]
    try:
        res = binding.batch_solve(plans, K)
        for (name, _, _), p, r, a in zip(inst, plans, res, alone):
            _same(_snapshot(p, r), a)
    finally:
        for p in plans:
            p.close()


def test_batch_from_different_pool_sizes_and_a_full_pool(torch):
    """Instances enter the batch at different pool sizes; one whose pool is full
    reports DAO_ESTATE and is left unchanged; the others continue exactly as a
    second dao_solve would."""
    from paper_1003_5402_gb300 import Plan, binding
    inst = _instances()[:4]
    pre = [0, 3, 5, 0]
    ref = []
    for (name, case, kw), k0 in zip(inst, pre):
        with Plan(case, **kw) as p:
            if k0:
                p.solve(k0)
            ref.append(_snapshot(p, p.solve(6)))
    plans = [Plan(case, **kw) for name, case, kw in inst]
    full = Plan(inst[0][1], k_max=2)
    try:
        for p, k0 in zip(plans, pre):
            if k0:
                p.solve(k0)
        full.solve(2)
        before = full.apertures()
        res = binding.batch_solve(plans + [full], 6)
        for p, r, a in zip(plans, res, ref):
            _same(_snapshot(p, r), a)
        assert res[-1][0] == binding.DAO_ESTATE and res[-1][1] == 2
        after = full.apertures()
        assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(before, after))
    finally:
        for p in plans + [full]:
            p.close()


def test_batch_rejects_bad_arguments(torch):
    from paper_1003_5402_gb300 import DaoError, Plan, binding
    case = P.make_case(P.spec_micro())
    with Plan(case) as p, Plan(case, use_graphs=0) as q:
        with pytest.raises(DaoError):
            binding.batch_solve([p, p], 3)          # listed twice
        with pytest.raises(DaoError):
            binding.batch_solve([p, q], 3)          # host-driven context
        assert binding.batch_solve([], 3) == []


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_choice_cache_and_parity(torch, tmp_path, prec):
    from paper_1003_5402_gb300 import Plan, binding
    case = P.make_case(P.spec_tiny())
    cache = str(tmp_path / "tune.txt")
    with Plan(case, precision=prec) as p:
        t1 = p.autotune(cache)
        assert not t1["from_cache"]
        assert t1["dose_lanes"] in ((4, 8, 16, 32) if prec == 0 else (4, 8, 16))
        assert t1["column_lanes"] in (0, 1, 2, 4, 8, 16) and t1["dt_threads"] in (64, 128, 256)
        assert t1["dose_form"] in ("lanes", "units") and t1["dt_map"] in ("grouped", "consecutive")
        x = np.random.default_rng(1).uniform(0.0, 2.0, size=case.n_beamlets).astype(np.float32)
        zd = torch.empty(case.n_voxels, dtype=torch.float32, device="cuda")
        p.k_dose(torch.from_numpy(x).cuda(), zd)
        z = zd.cpu().numpy().astype(np.float64)
        st, n, trace = p.solve(6)
        aps = p.apertures()
    if prec == 0:
        ref = O.dose(O.csr64(case), x.astype(np.float64))
        bound, m = sum_abs_rows(case, x)
        assert np.all(np.abs(z - ref) <= (m + 6) * U32 * bound + U32 * np.abs(ref))
        oref = O.column_generation(case, 6)
        assert all(a[0] == b[0] and np.array_equal(a[1], b[1]) for a, b in zip(aps, oref.apertures))
    with Plan(case, precision=prec) as p:
        t2 = p.autotune(cache)
    assert t2["from_cache"] and {k: t2[k] for k in t1 if k != "from_cache"} == \
        {k: t1[k] for k in t1 if k != "from_cache"}
    lines = open(cache).read().splitlines()
    forms = {"lanes": "1", "units": "2", "grouped": "1", "consecutive": "2"}
    assert len(lines) == 1 and lines[0].split()[1:] == [str(t1["dose_lanes"]), str(t1["column_lanes"]),
                                                       str(t1["dt_threads"]), forms[t1["dose_form"]],
                                                       forms[t1["dt_map"]]]


def test_batch_of_full_size_instances_against_the_oracle(torch):
    """Batched re-plans of the benchmark's sizes (a perturbed prostate-shaped
    instance in FP32, a perturbed H&N-shaped instance in FP16 storage, the
    small box) against the oracle: each instance alone passes the every-round
    oracle check of the free-running path, and the batch's result is bitwise
    that plan."""
    from paper_1003_5402_gb300 import Plan, binding
    from _helpers import quantized_case
    from test_gpu_cg import _free_running_checked
    K = 50
    inst = [(P.make_case(P.perturb(P.spec_prostate(), 4001)), {"precision": 0}),
            (P.make_case(P.perturb(P.spec_hn(), 4017)), {"precision": 1}),
            (P.make_case(P.spec_tiny()), {"precision": 0})]
    checked = []
    for case, kw in inst:
        ref_case = case if kw["precision"] == 0 else quantized_case(case, "fp16")
        checked.append(_free_running_checked(case, K, torch, plan_kw=kw, ref_case=ref_case))
    plans = [Plan(c, **kw) for c, kw in inst]
    try:
        res = binding.batch_solve(plans, K)
        for p, r, ref in zip(plans, res, checked):
            st, n, trace = r
            assert n == K
            aps = p.apertures()
            assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(aps, ref["apertures"]))
            assert np.array_equal(p.intensities(), ref["y"])
            z, F = p.dose()
            assert np.array_equal(z, ref["z"]) and F == ref["F"]
    finally:
        for p in plans:
            p.close()


def test_persistent_batch_equals_each_instance_alone_bitwise(torch):
    """dao_batch_solve_persistent (every round's master solves in one
    cooperative launch, a group of blocks per plan): each instance's results
    are bitwise those of solving it alone on that many blocks, for instances of
    different sizes, storage and MLC constraints, on two calls in a row (the
    second reuses the captured graph)."""
    from paper_1003_5402_gb300 import Plan, binding
    K = 12
    inst = _instances() + [("micro_interdig", P.make_case(P.spec_micro()),
                            {"mlc_constraint": binding.DAO_MLC_INTERDIGITATION})]
    GB = binding.load().dao_batch_group_size(len(inst), 0)
    assert GB >= 1
    alone = []
    for name, case, kw in inst:
        with Plan(case, master_blocks=GB, **kw) as p:
            alone.append(_snapshot(p, p.solve(K)))
    plans = [Plan(case, **kw) for name, case, kw in inst]
    try:
        for call in range(2):
            for p in plans:
                p.reset()
            res = binding.batch_solve(plans, K, persistent=True)
            for (name, _, _), p, r, a in zip(inst, plans, res, alone):
                _same(_snapshot(p, r), a)
    finally:
        for p in plans:
            p.close()


def test_persistent_batch_of_full_size_instances_against_the_oracle(torch):
    """The fused batch at the benchmark's sizes: a perturbed prostate-shaped
    instance (FP32), a perturbed H&N-shaped instance (FP16) and the small box;
    each plan alone on the batch's group size passes the every-round oracle
    check, and the batch's result is bitwise that plan."""
    from paper_1003_5402_gb300 import Plan, binding
    from _helpers import quantized_case
    from test_gpu_cg import _free_running_checked
    K = 50
    inst = [(P.make_case(P.perturb(P.spec_prostate(), 4002)), {"precision": 0}),
            (P.make_case(P.perturb(P.spec_hn(), 4018)), {"precision": 1}),
            (P.make_case(P.spec_tiny()), {"precision": 0})]
    GB = binding.load().dao_batch_group_size(len(inst), 0)
    checked = []
    for case, kw in inst:
        ref_case = case if kw["precision"] == 0 else quantized_case(case, "fp16")
        checked.append(_free_running_checked(case, K, torch, plan_kw=dict(kw, master_blocks=GB), ref_case=ref_case))
    plans = [Plan(c, **kw) for c, kw in inst]
    try:
        res = binding.batch_solve(plans, K, persistent=True)
        for p, r, ref in zip(plans, res, checked):
            assert r[1] == K
            aps = p.apertures()
            assert all(x[0] == y[0] and np.array_equal(x[1], y[1]) for x, y in zip(aps, ref["apertures"]))
            assert np.array_equal(p.intensities(), ref["y"])
            z, F = p.dose()
            assert np.array_equal(z, ref["z"]) and F == ref["F"]
    finally:
        for p in plans:
            p.close()

