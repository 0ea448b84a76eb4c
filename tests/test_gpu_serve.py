"""The re-plan server on the GPU: every result equals the same plan computed
alone with dao_solve (bitwise: objective, dose, intensities, apertures), plans
run concurrently, the admission footprint bounds the device memory a plan
really holds, and a memory budget that fits any one plan but no two admits one
plan at a time."""
import numpy as np
import pytest

import phantom as P
from _helpers import need_cuda, random_case

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]


@pytest.fixture(scope="module")
def torch():
    t = need_cuda()
    from paper_1003_5402_gb300 import build
    build.build()
    return t


def _cases():
    micro = P.spec_micro()
    return [P.make_case(micro), P.make_case(P.perturb(micro, 9001)), P.make_case(P.spec_tiny()),
            random_case(31, 3001, rows=[3, 5, 2], cols=[7, 5, 13], mean_row=9.0),
            P.make_case(P.perturb(micro, 9002))]


@pytest.mark.parametrize("solve_slots", [0, 1])
def test_server_results_equal_plans_alone(torch, solve_slots):
    """Every request's plan bitwise the plan alone, with all admitted plans'
    rounds on the GPU at once (solve_slots 0) and one plan's at a time in
    admission order (solve_slots 1)."""
    from paper_1003_5402_gb300 import Plan, Server
    cases = _cases()
    K = 10
    alone = []
    for c in cases:
        with Plan(c) as p:
            st, n, trace = p.solve(K)
            z, F = p.dose()
            aps = p.apertures()
            alone.append((st, n, F, z, p.intensities(), aps))
    with Server(max_slots=3, solve_slots=solve_slots) as s:
        ids = [s.submit(c, K) for c in cases]
        res = [s.wait(i, 120_000) for i in ids]
        stats = s.stats()
    for r, (st, n, F, z, y, aps) in zip(res, alone):
        assert r["status"] == st and r["n_apertures"] == n and r["error"] == ""
        assert r["objective"] == F and np.array_equal(r["dose"], z) and np.array_equal(r["y"], y)
        for k, (b, lv) in enumerate(aps):
            assert r["beams"][k] == b and np.array_equal(r["leaves"][k][: len(lv)], lv)
    assert stats["completed"] == len(cases) and stats["failed"] == 0 and stats["max_active"] >= 2


def test_server_full_size_results_against_the_oracle(torch):
    """Requests of the serving workload's sizes (a perturbed prostate-shaped
    instance and the small box, FP16 storage, 50 apertures) through the
    server, submitted together so that they run side by side: each result is
    bitwise the plan that passes the every-round oracle check of the
    free-running path."""
    from paper_1003_5402_gb300 import Server
    from _helpers import quantized_case
    from test_gpu_cg import _free_running_checked
    K = 50
    cases = [P.make_case(P.perturb(P.spec_prostate(), 9011)), P.make_case(P.perturb(P.spec_tiny(), 9003))]
    checked = [_free_running_checked(c, K, torch, plan_kw={"precision": 1}, ref_case=quantized_case(c, "fp16"))
               for c in cases]
    with Server(max_slots=4, precision=1) as s:
        ids = [s.submit(c, K) for c in cases]
        res = [s.wait(i, 120_000) for i in ids]
    for r, ref in zip(res, checked):
        assert r["status"] == 0 and r["n_apertures"] == K and r["error"] == ""
        assert r["objective"] == ref["F"] and np.array_equal(r["dose"], ref["z"]) and np.array_equal(r["y"], ref["y"])
        for k, (b, lv) in enumerate(ref["apertures"]):
            assert r["beams"][k] == b and np.array_equal(r["leaves"][k][: len(lv)], lv)


def test_footprint_bounds_the_device_memory_of_a_plan(torch):
    from paper_1003_5402_gb300 import Plan, Server, release_cached_memory
    case = P.make_case(P.spec_prostate())
    with Server(max_slots=1) as s:
        fp = s.footprint(case)
    torch.cuda.synchronize()
    # destroyed plans' memory stays in the library's pool: empty it, so that the
    # pool grows by this plan's peak (its build temporaries included)
    release_cached_memory(0)
    free0, _ = torch.cuda.mem_get_info()
    with Plan(case) as p:
        p.solve(2)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    used = free0 - free1
    assert used > 0 and fp >= used and fp <= 2 * used + (64 << 20), (fp, used)


def test_budget_of_one_footprint_runs_plans_one_at_a_time(torch):
    from paper_1003_5402_gb300 import Server
    cases = _cases()[:3]
    with Server(max_slots=3) as probe:
        fps = sorted(probe.footprint(c) for c in cases)
    budget = fps[-1]                              # every plan fits alone, no two together
    assert fps[0] + fps[1] > budget
    with Server(max_slots=3, hbm_budget_bytes=budget) as s:
        ids = [s.submit(c, 6) for c in cases]
        assert all(s.wait(i, 120_000)["status"] in (0, 1, 2) for i in ids)
        assert s.stats()["max_active"] == 1


def test_plans_created_from_several_threads_at_once(torch):
    """Plans of different sizes and storage created at the same time from
    several host threads (as the server's slots do): every one succeeds and
    plans the same as when created alone.  (Process-wide kernel attributes
    must never be set to one plan's own size.)"""
    import threading
    from paper_1003_5402_gb300 import Plan, binding
    cases = [(P.make_case(P.spec_micro()), {}), (P.make_case(P.spec_tiny()), {"precision": 1}),
             (random_case(33, 2000, rows=[4, 6], cols=[9, 30], mean_row=20.0), {}),
             (P.make_case(P.spec_micro()), {"mlc_constraint": binding.DAO_MLC_INTERDIGITATION}),
             (P.make_case(P.spec_tiny()), {"mlc_constraint": binding.DAO_MLC_JAWS})]
    alone = []
    for c, kw in cases:
        with Plan(c, **kw) as p:
            alone.append(p.solve(6)[2])
    out = [None] * (3 * len(cases))
    errs = []

    def work(i):
        try:
            c, kw = cases[i % len(cases)]
            with Plan(c, **kw) as p:
                out[i] = p.solve(6)[2]
        except Exception as e:  # noqa: BLE001 - reported below
            errs.append(repr(e))
    th = [threading.Thread(target=work, args=(i,)) for i in range(len(out))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for i, tr in enumerate(out):
        assert np.array_equal(tr, alone[i % len(cases)]), i
