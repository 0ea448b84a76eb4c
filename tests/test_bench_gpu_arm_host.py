"""The bench's GPU arm executed end to end on the host, with a stand-in torch
and a stand-in Plan in place of the CUDA calls: every line of the arm that does
not touch a GPU runs (clock sampler, timed loop bookkeeping, profiled plan and
roofline, SpMV records, mixed precision, e2e with page-locked inputs, JSON
assembly), and the printed line carries the contract's keys.  Batch, serve and
the oracle baseline are skipped (they are covered by their own tests)."""
import json
import sys
import types

import numpy as np


class _Event:
    clock = 0.0

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        _Event.clock += 1.0
        self.t = _Event.clock

    def elapsed_time(self, other):
        return 8.5 * (other.t - self.t)


class _Buf:
    def __init__(self, n):
        self.n = n

    def zero_(self):
        return self


class _HostTensor:
    def __init__(self, a):
        self.a = a

    def pin_memory(self):
        return _HostTensor(self.a.copy())

    def numpy(self):
        return self.a


def _fake_torch():
    cuda = types.SimpleNamespace(
        set_device=lambda d: None, current_device=lambda: 0, synchronize=lambda: None,
        current_stream=lambda: types.SimpleNamespace(cuda_stream=0), Event=_Event,
        get_device_name=lambda d: "stand-in")
    return types.SimpleNamespace(
        cuda=cuda, float32="float32", empty=lambda n, dtype=None, device=None: _Buf(n),
        rand=lambda n, device=None: _Buf(n), randn=lambda n, device=None: _Buf(n),
        empty_like=lambda b: _Buf(b.n), from_numpy=_HostTensor)


class _Plan:
    made = []

    def __init__(self, case, **kw):
        self.case, self.kw, self.k, self.launches = case, kw, 0, 0
        _Plan.made.append(self)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def close(self):
        pass

    def autotune(self, cache_path=None):
        return {"dose_lanes": 8, "column_lanes": 8, "dt_threads": 64, "dose_form": "units", "dt_map": "consecutive",
                "from_cache": False}

    def reset(self):
        self.k = 0

    def solve(self, n):
        self.k = n
        self.launches += 3 * n
        return 0, n, np.linspace(1.0, 0.5, n)

    def launch_count(self):
        return self.launches

    def master_stats(self):
        return np.full(self.k, 5, np.int32), np.ones(self.k, np.int32), np.zeros(self.k)

    def profile_enable(self, on=True):
        pass

    def profile_read(self, kc):
        return (self.k, 0.14 * self.k) if kc == "master_solve" else (self.k, 0.01 * self.k)

    def k_time(self, kc, K=0, reps=20):
        return 7.0

    def k_dose(self, x, z, g=None, objective=True):
        return None

    def k_beamlet_prices(self, pi, w):
        pass

    def k_time_cold(self, kc, flush, reps=20):
        return {"dose": 22.5, "dt": 19.5}[kc]

    def dose(self):
        return np.zeros(self.case.n_voxels, np.float32), 0.5


def test_gpu_arm_runs_on_stand_ins_and_prints_the_contract_line(monkeypatch, capsys, tmp_path):
    import bench
    import paper_1003_5402_gb300 as pkg
    from paper_1003_5402_gb300 import build
    monkeypatch.setitem(sys.modules, "torch", _fake_torch())
    monkeypatch.setattr(pkg, "Plan", _Plan)
    monkeypatch.setattr(build, "build", lambda *a, **k: None)
    monkeypatch.setattr(bench, "strip_case", lambda case: case)   # no device generation here
    monkeypatch.setenv("PATH", str(tmp_path))            # no nvidia-smi: the clock record is null
    monkeypatch.setenv("DAO_BENCH_CLOCKS_DIR", str(tmp_path))
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--config", "tiny", "--apertures", "4", "--steps", "2",
                                      "--warmup", "3", "--skip-cpu", "--skip-batch", "--skip-serve"])
    _Plan.made.clear()
    bench.main()
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
                "clocks", "gpu_launches"):
        assert key in d, key
    assert d["metric"] == "ms per 4-aperture plan" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] == 8.5 and d["gpu_launches"] == 2 * 3 * 4
    assert d["config"]["apertures"] == 4 and d["config"]["workload"].startswith("small box FP32")
    assert d["config"]["storage"] == "fp32"
    r = d["roofline"]
    assert r["kernel"] == "k_master_persist" and r["unit"] == "GB/s" and 0 < r["frac"] < 10
    assert r["l2"]["us_per_evaluation"] > 0 and r["l2"]["slab_gbs"] > 0
    assert set(d["spmv"]) == {"fp32", "fp16"} and d["spmv"]["fp32"]["dose"]["us"] == 22.5
    assert d["spmv"]["fp32"]["form"]["dose"] == "units" and d["spmv"]["fp32"]["form"]["dt_map"] == "consecutive"
    st = d["spmv_strip_profile"]
    assert set(st) == {"nnz", "nnz_gauss", "fp32", "fp16"} and st["fp16"]["dt"]["us"] == 19.5
    assert d["mixed_precision"]["other_ms_per_plan"] == 8.5
    e = d["e2e"]
    assert e["inputs"] == "page-locked host arrays" and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["clocks"] is None and d["cpu_baseline"] is None
    # the e2e plans were built from the page-locked copies, not from the case itself
    e2e_plans = [p for p in _Plan.made if hasattr(p.case, "pinned_tensors")]
    assert len(e2e_plans) == min(2, 3) + 1          # e2e steps + one warm-up plan
