"""The re-plan server's scheduler on the host, in its simulation mode (no CUDA
call, requests "run" for a fixed time per aperture): admission by slots and by
the device-memory budget, arrival order, a request that can never fit, an
invalid request, a full queue, a timed-out wait, concurrent submitters and
shutdown with queued work.  Failures are made on the host (invalid inputs,
budgets, timeouts); nothing here touches a GPU."""
import threading
import time

import numpy as np
import pytest

import phantom as P
from _helpers import random_case

pytestmark = pytest.mark.timeout(60)


@pytest.fixture(scope="module")
def lib():
    from paper_1003_5402_gb300 import build
    build.build()
    from paper_1003_5402_gb300 import binding
    return binding.load()


@pytest.fixture(scope="module")
def small():
    return random_case(7, 400, rows=[2, 3], cols=[4, 5], mean_row=6.0)


@pytest.fixture(scope="module")
def big():
    return random_case(8, 100000, rows=[4, 4], cols=[8, 8], mean_row=40.0)


def _server(**kw):
    from paper_1003_5402_gb300 import Server
    kw.setdefault("simulate_ms_per_aperture", 1.0)
    kw.setdefault("hbm_budget_bytes", 64 << 30)
    return Server(**kw)


def test_requests_complete_with_latency_accounting(lib, small):
    with _server(max_slots=2) as s:
        ids = [s.submit(small, 5) for _ in range(6)]
        res = [s.wait(i, 10_000) for i in ids]
        st = s.stats()
    for r in res:
        assert r["status"] == 0 and r["n_apertures"] == 5 and np.isnan(r["objective"])
        assert r["run_ms"] >= 4.0 and r["latency_ms"] >= r["run_ms"] and r["queue_ms"] >= 0.0
        assert abs(r["latency_ms"] - r["queue_ms"] - r["run_ms"]) < 1.0
    assert st["submitted"] == 6 and st["completed"] == 6 and st["failed"] == 0
    assert 1 <= st["max_active"] <= 2 and st["active"] == 0 and st["bytes_in_use"] == 0


def test_arrival_order_with_one_slot(lib, small):
    with _server(max_slots=1) as s:
        ids = [s.submit(small, 3) for _ in range(5)]
        res = {i: s.wait(i, 10_000) for i in ids}
    done_at = [res[i]["queue_ms"] for i in ids]
    assert all(a < b for a, b in zip(done_at, done_at[1:]))      # admitted in submission order


def test_solve_slots_queue_rounds_in_admission_order(lib, small):
    """solve_slots 1: four slots admit and create at once, but the plans' rounds
    (5 ms each in simulation) take the GPU one plan at a time, in admission
    order; without it the four run side by side."""
    import time
    with _server(max_slots=4, solve_slots=1, simulate_ms_per_aperture=1.0) as s:
        t0 = time.perf_counter()
        ids = [s.submit(small, 5) for _ in range(6)]
        res = [s.wait(i, 10_000) for i in ids]
        span = 1e3 * (time.perf_counter() - t0)
        st = s.stats()
    assert all(r["status"] == 0 for r in res) and st["max_active"] == 4
    assert span >= 6 * 5.0 - 1.0                                   # the six solves one after another
    lat = [r["latency_ms"] for r in res]
    assert all(b > a for a, b in zip(lat, lat[1:]))                 # finished in admission order
    assert res[0]["gpu_wait_ms"] < 2.0 and res[2]["gpu_wait_ms"] >= 2 * 5.0 - 1.0
    with _server(max_slots=4, simulate_ms_per_aperture=1.0) as s:
        t0 = time.perf_counter()
        ids = [s.submit(small, 5) for _ in range(4)]
        res = [s.wait(i, 10_000) for i in ids]
        span = 1e3 * (time.perf_counter() - t0)
    assert span < 4 * 5.0 and all(r["gpu_wait_ms"] < 2.0 for r in res)


def test_memory_budget_admits_one_plan_at_a_time(lib, small):
    with _server(max_slots=4) as probe:
        fp = probe.footprint(small)
    with _server(max_slots=4, hbm_budget_bytes=int(1.5 * fp)) as s:
        ids = [s.submit(small, 4) for _ in range(4)]
        for i in ids:
            assert s.wait(i, 10_000)["status"] == 0
        assert s.stats()["max_active"] == 1


def test_request_that_can_never_fit_is_rejected_not_blocking(lib, small, big):
    with _server(max_slots=2) as probe:
        fs, fb = probe.footprint(small), probe.footprint(big)
    assert fb > 2 * fs
    with _server(max_slots=2, hbm_budget_bytes=(fs + fb) // 2) as s:
        a = s.submit(big, 3)
        b = s.submit(small, 3)
        ra, rb = s.wait(a, 10_000), s.wait(b, 10_000)
        st = s.stats()
    from paper_1003_5402_gb300 import binding
    assert ra["status"] == binding.DAO_ENOMEM and "exceeds" in ra["error"]
    assert rb["status"] == 0 and st["rejected"] == 1 and st["completed"] == 1


def test_invalid_request_fails_and_others_continue(lib, small):
    from paper_1003_5402_gb300 import binding
    bad = random_case(7, 400, rows=[2, 3], cols=[4, 5], mean_row=6.0)
    bad.over_w = bad.over_w.copy()
    bad.over_w[0] = -1.0                                            # weights must be >= 0
    with _server(max_slots=2) as s:
        i1 = s.submit(small, 2)
        i2 = s.submit(bad, 2)
        i3 = s.submit(small, 2)
        r2 = s.wait(i2, 10_000)
        assert r2["status"] == binding.DAO_EINVAL and "weights" in r2["error"]
        assert s.wait(i1, 10_000)["status"] == 0 and s.wait(i3, 10_000)["status"] == 0
        st = s.stats()
    assert st["failed"] == 1 and st["completed"] == 2


def test_full_queue_and_timed_out_wait(lib, small):
    from paper_1003_5402_gb300 import DaoError, binding
    with _server(max_slots=1, queue_capacity=2, simulate_ms_per_aperture=20.0) as s:
        a = s.submit(small, 5)                                     # 100 ms
        time.sleep(0.02)                                           # admitted: the queue is empty again
        b = s.submit(small, 1)
        c = s.submit(small, 1)
        with pytest.raises(DaoError) as e:
            s.submit(small, 1)
        assert e.value.status == binding.DAO_EBUSY
        with pytest.raises(DaoError) as e:
            s.wait(a, 1.0)
        assert e.value.status == binding.DAO_ETIMEOUT
        assert s.poll(b) is None
        for i in (a, b, c):
            assert s.wait(i, 10_000)["status"] == 0
        with pytest.raises(DaoError):
            s.poll(a)                                              # reported once


def test_concurrent_submitters(lib, small):
    with _server(max_slots=3, simulate_ms_per_aperture=0.2) as s:
        out, lock = [], threading.Lock()

        def client():
            mine = [s.submit(small, 3) for _ in range(10)]
            got = [s.wait(i, 20_000)["status"] for i in mine]
            with lock:
                out.extend(got)

        ts = [threading.Thread(target=client) for _ in range(4)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        st = s.stats()
    assert out == [0] * 40 and st["completed"] == 40 and st["max_active"] <= 3


def test_shutdown_with_queued_work_returns(lib, small):
    s = _server(max_slots=1, simulate_ms_per_aperture=10.0)
    for _ in range(5):
        s.submit(small, 5)
    t0 = time.perf_counter()
    s.close()                                                      # running plan drains, the rest is cancelled
    assert time.perf_counter() - t0 < 5.0


def test_server_options_are_validated(lib):
    from paper_1003_5402_gb300 import DaoError
    with pytest.raises(DaoError):
        _server(max_slots=0)
    with pytest.raises(DaoError):
        _server(hbm_budget_bytes=0)                                # simulation needs a budget
    with pytest.raises(DaoError):
        _server(solve_slots=-1)
