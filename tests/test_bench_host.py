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


class _Op:
    def __init__(self, g):
        self.nx, self.ny, self.D = g.nx, g.ny, g.nx * g.ny


class _Ctx:
    closed = 0

    def set_graphs(self, on):
        pass

    def set_basis_storage(self, s):
        pass

    def close(self):
        _Ctx.closed += 1


class _FakeLib:
    """Stands in for the CUDA library: records the queue calls."""
    Context = _Ctx

    def __init__(self):
        self.calls = []

    def fdfd_operator(self, g, eps):
        return _Op(g)

    def fdfd_source(self, op, i, s, j):
        return object()

    def gmres_solve_queue(self, lanes, A, b, U=None, width=64, tol=1e-6, restart=200, maxit=5000,
                          precision="c64"):
        self.calls.append((len(lanes), width, restart, len(A)))
        return None, [{"converged": 1, "iters": 1000 + restart, "true_rel_residual": 5e-7} for _ in A], 0


class _FakeTorch:
    class cuda:
        @staticmethod
        def synchronize():
            pass

    @staticmethod
    def as_tensor(x, device=None):
        return x


def test_queue_line_tunes_width_lanes_and_restart_with_a_fake_library():
    import argparse
    from paper_1902_00090_gb300 import autotune, inputs
    lib = _FakeLib()
    args = argparse.Namespace(graphs="on", basis="f16", precision="c64", restart=200)
    _Ctx.closed = 0
    q = bench.queue_line(lib, autotune, inputs, _FakeTorch, "cpu", args)
    assert q["converged"] == 64 and q["unit"] == "solves/s" and q["value"] > 0
    assert q["tuned"]["restart"] in (100, 200) and q["tuned"]["lanes"] in (1, 2)
    assert len(q["tuning"]) == 6 and {t["restart"] for t in q["tuning"]} == {100, 200}
    assert q["single_batch_value"] is not None
    # warm-up (2), tuning (6) and the timed run (1); every call sees the 64 solves
    assert len(lib.calls) == 9 and all(c[3] == 64 for c in lib.calls)
    assert _Ctx.closed == 2
