"""Host-side arithmetic of bench.py that needs no GPU: the clock record taken
from nvidia-smi samples, the DRAM-traffic records keyed by the kernel sources
and the grid, and the FP64-pipe roofline of the L2-resident workload.
"""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


class _FakeThread:
    def join(self, timeout=None):
        pass


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc, s._t, s.lines = _FakeProc(), _FakeThread(), list(lines)
    return s


def test_clock_record_median_max_and_active_reasons():
    # fields: sm, max sm, power, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = [
        "2070, 2070, 1100.5, Not Active, Not Active, Not Active, Not Active",
        "1980, 2070, 1390.2, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 1200.0, Not Active, Not Active, Not Active, Not Active",  # unreadable
        "garbled line",
    ]
    rec = _sampler(lines).stop()
    assert rec == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}


def test_clock_record_reports_every_slowdown_reason():
    lines = ["1500, 2070, 900, Active, Active, Active, Not Active",
             "1400, 2070, 900, Not Active, Not Active, Not Active, Not Active"]
    rec = _sampler(lines).stop()
    assert rec["sm_mhz"] == 1450.0
    assert rec["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_record_without_samples_is_none():
    assert _sampler([]).stop() is None
    assert bench.ClockSampler(0).stop() is None  # never started


def test_traffic_record_needs_matching_sources_and_grid(tmp_path, monkeypatch):
    rec = {"kernel_hash": "abc123", "grid": [256, 256, 256], "dram_bytes_per_launch": 1.5e9}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "t.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: "abc123")
    assert bench.recorded_traffic("t.json", (256, 256, 256)) == 1.5e9
    assert bench.recorded_traffic("t.json", (128, 128, 128)) is None  # another size
    assert bench.recorded_traffic("missing.json", (256, 256, 256)) is None
    monkeypatch.setattr(bench, "kernel_hash", lambda: "changed")
    assert bench.recorded_traffic("t.json", (256, 256, 256)) is None  # sources changed


def test_kernel_hash_covers_every_kernel_header():
    csrc = os.path.join(ROOT, "paper_1808_06787_gb300", "csrc")
    headers = sorted(f for f in os.listdir(csrc) if f.endswith(".cuh"))
    assert [os.path.basename(p) for p in bench.KERNEL_SOURCES] == headers
    assert len(bench.kernel_hash()) == 16


def test_fp64_roofline_arithmetic():
    wl = bench.make_workload("sine", 256)
    assert wl.grid == (128, 128, 1) and wl.cells == 128 * 128
    step_ms = 0.006
    r = bench.fp64_roofline(wl, step_ms, 152, 2070.0)
    flops = 152.0 * 128 * 128
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["algorithmic_flops_per_launch"] == pytest.approx(flops)
    assert r["achieved"] == pytest.approx(flops / (step_ms * 1e-3) / 1e12, rel=1e-3)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.07e9 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)


def test_job_rate_counts_the_units_of_all_ranks():
    assert bench.job_rate(1000.0, 4, 2.0) == pytest.approx(2.0e6)


def test_fp64_peak_follows_sm_count_and_sampled_clock():
    assert bench.fp64_peak_tflops(148, 1900.0) == pytest.approx(148 * 2 * 2 * 1.9e9 / 1e12)
    wl = bench.make_workload("sine", 256)
    r = bench.fp64_roofline(wl, 0.006, 148, 1900.0)
    assert r["peak"] == pytest.approx(148 * 2 * 2 * 1.9e9 / 1e12, rel=1e-3)
    assert "148 SMs" in r["peak_source"] and "1900 MHz" in r["peak_source"]


def test_sharded_grid_stacks_one_workload_grid_per_rank():
    assert bench.sharded_grid(bench.make_workload("tube", 256), 4) == (256, 256, 1024)
    assert bench.sharded_grid(bench.make_workload("blobs", 256), 2) == (2048, 4096, 1)
    assert bench.sharded_grid(bench.make_workload("line", 256), 8) == (8 << 26, 1, 1)
    assert bench.sharded_grid(bench.make_workload("tube", 256), 1) == (256, 256, 256)
