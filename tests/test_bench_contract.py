"""bench.py's host-side contract, without a GPU: the reference arm's JSON line (the oracle timed
on the host cores, on a small workload here) and the parsing of the clock samples that decide
which throttle reasons the bench line reports."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "square-p2-20x20-expsep", "--steps", "2", "--warmup", "1"],
                         check=True, capture_output=True, text=True, cwd=ROOT, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is False
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "square-p2-20x20-expsep" and d["config"]["Ntilde"] == 484


class _FakeProc:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _clocks(text):
    c = bench.ClockSampler(0)
    c.proc = _FakeProc(text)
    return c.stop()


def test_clock_samples_median_and_reasons():
    text = "\n".join([
        "2070, 2070, 900.1, Not Active, Not Active, Not Active, Not Active",
        "2040, 2070, 1200.5, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1300.0, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, 10.0, Not Active, Not Active, Not Active, Not Active",   # skipped
        "garbage line",
    ])
    r = _clocks(text)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]


def test_clock_samples_report_thermal_slowdown():
    r = _clocks("1500, 2070, 1400, Not Active, Active, Active, Not Active\n")
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
