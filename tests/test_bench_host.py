"""Host-side logic of bench.py on CPU: the clock sampler's time window, the ncu records and the
issue roofline arithmetic (no GPU, no nvidia-smi: a stand-in script prints sample lines)."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

FAKE_SMI = r"""#!/usr/bin/env python3
# prints one CSV sample line every 50 ms, like nvidia-smi --query-gpu ... -lms 50
import datetime, os, time
reason = "Active" if os.environ.get("FAKE_SMI_POWER_CAP") else "Not Active"
while True:
    ts = datetime.datetime.now().strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    print("%s, 0, 1980, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, %s" % (ts, reason), flush=True)
    time.sleep(0.05)
"""


@pytest.fixture
def fake_smi(tmp_path, monkeypatch):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE_SMI)
    p.chmod(p.stat().st_mode | stat.S_IEXEC | stat.S_IXGRP | stat.S_IXOTH)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    return p


def test_clock_sampler_keeps_samples_inside_the_window(fake_smi):
    s = bench.ClockSampler(0)
    assert s.proc is not None and os.path.getsize(s.path) > 0  # the first sample came before the region
    time.sleep(0.2)
    t0 = time.time()
    time.sleep(0.4)
    t1 = time.time()
    out = s.stop((t0, t1))
    assert out["sm_mhz"] == 1980.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []
    # 50 ms sampling over a 0.4 s window: about 8 samples, none from before or after it
    assert 4 <= out["samples"] == out["samples_in_timed_region"] <= 10


def test_clock_sampler_reports_throttle_reasons(fake_smi, monkeypatch):
    monkeypatch.setenv("FAKE_SMI_POWER_CAP", "1")
    s = bench.ClockSampler(0)
    t0 = time.time()
    time.sleep(0.2)
    out = s.stop((t0, time.time()))
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_window_without_samples_falls_back_to_the_nearest(fake_smi):
    s = bench.ClockSampler(0)
    time.sleep(0.3)
    t = time.time()
    out = s.stop((t, t))  # an empty window (shorter than the sampling interval)
    assert out["samples_in_timed_region"] == 0 and out["samples"] == 2


def test_profile_records_follow_the_kernel_sources(monkeypatch, tmp_path):
    h = bench.kernel_source_hash()
    rec = tmp_path / "launches.md"
    rec.write_text("text\n\ntraffic_record: kernel=vpass sources=%s bytes_per_launch=1341341952\n"
                   "instr_record: kernel=vpass sources=%s thread_inst_per_launch=9715365121\n" % (h, h))
    monkeypatch.setattr(bench, "PROFILE_LAUNCHES", str(rec))
    assert bench.recorded_traffic("vpass_solve") == 1341341952
    assert bench.recorded_instructions("vpass_solve") == 9715365121
    assert bench.recorded_traffic("hpass") is None  # no record for that kernel
    # any other source hash (a kernel changed since the capture) voids them
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("vpass_solve") is None
    assert bench.recorded_instructions("vpass_solve") is None
    assert bench.issue_roofline("vpass_solve", 0.35, {"sm_mhz": 2070.0}, 152) is None
    monkeypatch.setattr(bench, "PROFILE_LAUNCHES", str(tmp_path / "missing.md"))
    assert bench.recorded_traffic("vpass_solve") is None


def test_issue_roofline_arithmetic(monkeypatch):
    monkeypatch.setattr(bench, "recorded_instructions", lambda stage: 4_000_000_000)
    r = bench.issue_roofline("vpass_solve", 0.25, {"sm_mhz": 2000.0}, 100)
    assert r["bound"] == "alu" and r["unit"] == "Tinst/s"
    assert r["peak"] == pytest.approx(100 * 128 * 2000e6 / 1e12)  # 25.6 T/s
    assert r["achieved"] == pytest.approx(4e9 / 0.25e-3 / 1e12)   # 16 T/s
    assert r["frac"] == pytest.approx(16 / 25.6)
    # without a sampled clock the recipe's maximum SM clock stands in
    assert bench.issue_roofline("vpass_solve", 0.25, None, 100)["sm_mhz"] == 2070.0


class _FakeNvml:
    """Stands in for bench._Nvml: a fixed SM clock and the throttle-reason bits the test sets."""

    bits = 0

    def __init__(self, uuid, pci_bus_id, index):
        self.max_mhz = 2070.0

    def sample(self):
        return (1995.0, 800.0, _FakeNvml.bits)

    def close(self):
        pass


def test_nvml_sampler_every_2ms_inside_the_window(monkeypatch):
    monkeypatch.setattr(bench, "_Nvml", _FakeNvml)
    _FakeNvml.bits = 0
    s = bench.ClockSampler(0)
    assert s.nvml is not None and s.source.startswith("nvml")
    time.sleep(0.05)
    t0 = time.time()
    time.sleep(0.1)
    t1 = time.time()
    out = s.stop((t0, t1))
    assert out["sm_mhz"] == 1995.0 and out["sm_max_mhz"] == 2070.0 and out["reasons"] == []
    # 2 ms sampling over a 0.1 s window: tens of samples, all inside it
    assert 20 <= out["samples"] == out["samples_in_timed_region"] <= 60


def test_nvml_sampler_decodes_throttle_bits(monkeypatch):
    monkeypatch.setattr(bench, "_Nvml", _FakeNvml)
    _FakeNvml.bits = 0x4 | 0x8 | 0x1  # power cap, hardware slowdown, idle (not a throttle reason kept)
    s = bench.ClockSampler(0)
    t0 = time.time()
    time.sleep(0.05)
    out = s.stop((t0, time.time()))
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
