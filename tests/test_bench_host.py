"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region (parsing of nvidia-smi samples)."""
import os
import sys
import threading

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


class FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def sampler_with(lines):
    c = bench.ClockSampler(0)
    c.proc = FakeProc()
    c.t = threading.Thread(target=lambda: None)
    c.t.start()
    c.lines = list(lines)
    return c


def test_clock_record_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    r = sampler_with(lines).stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_flags_throttling_and_missing_samples():
    r = sampler_with(["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"]).stop()
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["sm_mhz"] == 1500.0
    assert sampler_with([]).stop()["reasons"] == ["no samples"]
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
