"""The bench's clock sampler on the host, against a stand-in nvidia-smi on PATH
that prints one timestamped CSV sample every 10 ms in nvidia-smi's query format:
samples inside the timed region are the ones summarised, throttle reasons are
collected, and a region shorter than the sampling period falls back to the
warm-up and timed samples and says so."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = r'''#!{python}
import datetime, sys, time
mhz = {mhz}
thermal = "{thermal}"
while True:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    sys.stdout.write(f"0, {{mhz}}, 2070, 900.5, 0x0, Not Active, Not Active, {{thermal}}, Not Active, {{ts}}\n")
    sys.stdout.flush()
    time.sleep({period})
'''


def _fake_smi(tmp_path, monkeypatch, mhz=2070, thermal="Not Active", period=0.01):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text(FAKE.format(python=sys.executable, mhz=mhz, thermal=thermal, period=period))
    f.chmod(f.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", f"{d}{os.pathsep}{os.environ['PATH']}")
    monkeypatch.setenv("DAO_BENCH_CLOCKS_DIR", str(tmp_path / "clocks"))


def test_samples_inside_the_timed_region(tmp_path, monkeypatch):
    import bench
    _fake_smi(tmp_path, monkeypatch, mhz=1980)
    s = bench.ClockSampler(0)
    s.wait_first_sample()
    time.sleep(0.05)
    s.timed(True)
    time.sleep(0.3)
    s.timed(False)
    c = s.stop()
    assert c is not None and c["scope"] == "timed region"
    assert c["samples"] >= 5 and c["sm_mhz"] == 1980 and c["sm_max_mhz"] == 2070 and c["reasons"] == []
    assert os.path.exists(os.path.join(str(tmp_path / "clocks"), "dao_bench_clocks_rank0.csv"))


def test_throttle_reason_is_reported(tmp_path, monkeypatch):
    import bench
    _fake_smi(tmp_path, monkeypatch, thermal="Active")
    s = bench.ClockSampler(0)
    s.wait_first_sample()
    s.timed(True)
    time.sleep(0.2)
    s.timed(False)
    assert s.stop()["reasons"] == ["sw_thermal_slowdown"]


def test_short_region_falls_back_to_the_loaded_samples(tmp_path, monkeypatch):
    import bench
    _fake_smi(tmp_path, monkeypatch, period=0.2)
    s = bench.ClockSampler(0)
    s.wait_first_sample()
    time.sleep(0.5)              # the warm-up
    s.timed(True)
    s.timed(False)               # a timed region far shorter than the period
    c = s.stop()
    assert c is not None and c["scope"].startswith("warm-up and timed region") and c["samples"] >= 1


def test_no_nvidia_smi_gives_none(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    monkeypatch.setenv("DAO_BENCH_CLOCKS_DIR", str(tmp_path / "clocks"))
    s = bench.ClockSampler(0)
    s.wait_first_sample(limit_s=0.1)
    s.timed(True)
    s.timed(False)
    assert s.stop() is None


def test_unreadable_timestamps_keep_every_sample(tmp_path, monkeypatch):
    import bench
    _fake_smi(tmp_path, monkeypatch, mhz=2000)
    monkeypatch.setattr(bench.ClockSampler, "TS_FORMAT", "%d.%m.%Y")
    s = bench.ClockSampler(0)
    s.wait_first_sample()
    s.timed(True)
    time.sleep(0.1)
    s.timed(False)
    c = s.stop()
    assert c["scope"].startswith("every sample") and c["sm_mhz"] == 2000 and c["samples"] >= 1
