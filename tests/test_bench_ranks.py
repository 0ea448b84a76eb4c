"""The multi-GPU path of bench.py on the host: replicas only, so the ranks
exchange nothing but the timing.  Two gloo ranks on the CPU check that every
rank gets the slowest rank's time, that the whole-job time per plan divides it
by steps x ranks, and that under torchrun only rank 0 of the reference arm
does any work.  On one rank the reference arm's line carries the contract's
keys, and the SpMV bandwidth record is assembled from a stand-in plan."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

pytestmark = pytest.mark.timeout(120)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, local_ms, steps, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dist.barrier()
        total = bench.max_over_ranks(local_ms[rank], ws, "cpu")
        out.put((rank, total, bench.whole_job_ms_per_plan(total, steps, ws)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    local_ms = [120.0, 95.5]
    steps = 10
    procs = [ctx.Process(target=_rank, args=(r, 2, port, local_ms, steps, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=90) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, total, per_plan in res:
        assert total == 120.0
        assert per_plan == pytest.approx(120.0 / (steps * 2))


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.whole_job_ms_per_plan(80.0, 10, 1) == 8.0


def test_reference_arm_other_ranks_do_nothing(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "oracle_plan_seconds", lambda *a, **k: called.append(a) or 0.0)
    bench.run_reference(argparse.Namespace(config="tiny", apertures=5, steps=1, warmup=3, gpus=2))
    assert called == [] and capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    """Rank 0 of the reference arm times the oracle on the host and prints one
    JSON line with the keys of the bench contract (tiny workload, 4 apertures)."""
    import argparse
    import json

    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    bench.run_reference(argparse.Namespace(config="tiny", apertures=4, steps=1, warmup=3, gpus=1, precision="fp32"))
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "ms per 4-aperture plan" and d["unit"] == "ms"
    assert d["higher_is_better"] is False and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    assert d["config"]["workload"].startswith("small box FP32") and d["config"]["apertures"] == 4
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_spmv_bandwidth_record_from_a_stand_in_plan():
    """The SpMV record's arithmetic: algorithmic bytes over the cold median
    time, as a fraction of the measured copy peak and of the nominal HBM rate."""
    import types

    import numpy as np

    import bench
    case = types.SimpleNamespace(n_voxels=1000, n_beamlets=100, n_beams=4, nnz=50_000)
    fake_torch = types.SimpleNamespace(rand=lambda n, device=None: np.zeros(n, np.float32),
                                       randn=lambda n, device=None: np.zeros(n, np.float32),
                                       empty=lambda n, device=None: np.zeros(n, np.float32),
                                       empty_like=lambda a: np.zeros_like(a))
    calls = []
    plan = types.SimpleNamespace(k_dose=lambda x, z, g, objective=True: calls.append("dose"),
                                 k_beamlet_prices=lambda pi, w: calls.append("dt"),
                                 k_time_cold=lambda kc, flush, reps=20: {"dose": 2.0, "dt": 4.0}[kc])
    out = bench.spmv_bandwidth(fake_torch, plan, case, "fp32", None, 5000.0)
    assert calls == ["dose", "dt"]
    b_dose = 8 * 50_000 + 4 * 1001 + 4 * 100 + 4 * 1000 + 1000
    assert out["dose"]["bytes"] == b_dose and out["dose"]["us"] == 2.0
    assert out["dose"]["gbs"] == round(b_dose / 2e-6 / 1e9, 1)
    assert out["dose"]["frac_of_hbm"] == round(b_dose / 2e-6 / 1e9 / 5000.0, 4)
    assert out["dose"]["frac_of_nominal"] == round(b_dose / 2e-6 / 1e9 / bench.HBM_NOMINAL_GBS, 4)
    b_dt = 8 * 50_000 + 4 * 101 + 4 * 1000 + 4 * 100
    assert out["dt"]["bytes"] == b_dt and out["dt"]["us"] == 4.0


def test_pinned_inputs_keep_every_array_dao_create_reads():
    """The e2e leg's page-locked copy of a case: every array dao_create reads,
    equal to the original, with the dtype the binding passes through without a
    further copy (so the pointers it hands over are the page-locked ones)."""
    import types

    import numpy as np

    import bench
    import phantom
    from paper_1003_5402_gb300 import binding
    case = phantom.make_case(phantom.spec_micro())

    class _T:
        def __init__(self, a):
            self.a = a

        def pin_memory(self):
            return _T(self.a.copy())

        def numpy(self):
            return self.a

    c = bench.pinned_inputs(types.SimpleNamespace(from_numpy=_T), case)
    for name in ("indptr", "indices", "data", "rows", "cols", "voxel_struct", "is_target", "under_w", "under_t",
                 "over_w", "over_t"):
        assert np.array_equal(getattr(c, name), getattr(case, name)), name
    assert len(c.pinned_tensors) == 11
    D, g, s, w, rx, keep = binding._case_structs(c)
    assert keep[0] is c.indptr and keep[1] is c.indices and keep[2] is c.data and keep[5] is c.voxel_struct
    assert D.n_voxels == case.n_voxels and D.nnz == int(case.indptr[-1])


def test_one_thread_oracle_timing_runs_in_a_child():
    """The 1-thread oracle figure: a child interpreter with every thread count
    at 1 times a short plan of the small workload and reports seconds."""
    import bench
    secs = bench.oracle_plan_seconds_one_thread("tiny", 2, timeout_s=120)
    assert secs is not None and 0.0 < secs < 120.0
    assert bench.oracle_plan_seconds_one_thread("no-such-workload", 2, timeout_s=60) is None
