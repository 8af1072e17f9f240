"""CPU tests of bench.py's host logic: the clock record taken during the
timed region (median SM clock, maximum, throttle reasons parsed from
nvidia-smi's CSV) and the roofline constants' arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(tmp_path, rows):
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler(None)
    s.proc, s.path = _Proc(), str(p)
    return s


def test_clock_record_no_reason(tmp_path):
    rows = ["2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"] * 3 + \
           ["1965, 2070, 1000.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"]
    c = _sampler(tmp_path, rows).stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["reasons"] == [] and c["samples"] == 4


def test_clock_record_reasons(tmp_path):
    rows = ["1800, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            "1700, 2070, 1400.0, 0x0000000000000048, Not Active, Active, Not Active, Not Active",
            "[N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active",
            "short, row"]
    c = _sampler(tmp_path, rows).stop()
    assert c["sm_mhz"] == 1750.0                       # median of the numeric samples
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert c["samples"] == 3


def test_clock_record_without_samples(tmp_path):
    assert _sampler(tmp_path, [""]).stop()["reasons"] == ["no samples"]
    s = bench.ClockSampler(None)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_work_per_point_matches_its_parts():
    """Algorithmic work per located point (FP64 form: seed + K iterations;
    mixed: FP64 residual + basis, FP32 seed + K iterations + two compensated
    residuals) and the FP32 peak from the unit counts."""
    assert bench.WORK["fp64"]["f64"] == pytest.approx(4.1e3 + 3.43 * 8.4e3)
    assert bench.WORK["fp64"]["f32"] == 0.0
    assert bench.WORK["mixed"]["f64"] == pytest.approx(3.5e3 + 0.3e3)
    assert bench.WORK["mixed"]["f32"] == pytest.approx(4.1e3 + 3.43 * 8.4e3 + 2 * 19.3e3)
    assert bench.P32_NOMINAL == pytest.approx(152 * 128 * 2 * 2.07e9)
    # the value-only FP64 residual: 3 coordinates x (n^3 + n^2 + n) FMA at n = 8, 2 flops each
    assert bench.RESID == pytest.approx(2 * 3 * (8 ** 3 + 8 ** 2 + 8), rel=0.01)


def test_oracle_one_core_timing_restores_threads():
    """The one-core oracle timing runs on one thread and gives the thread
    count back; its results are the all-core oracle's (threads change only
    the schedule)."""
    import numpy as np

    import oracle
    import synth
    mesh, q = synth.cube4_small()
    n0 = oracle.num_threads()
    rate, m, dt = bench.oracle_rate_one_core(mesh, q, 0.2)
    assert rate > 0 and 1 <= m <= q.P and dt > 0
    assert oracle.num_threads() == n0
    oracle.set_threads(1)
    try:
        one = oracle.find(mesh.coords, mesh.N, mesh.sub, q.pts[:, :500])
    finally:
        oracle.set_threads(n0)
    allc = oracle.find(mesh.coords, mesh.N, mesh.sub, q.pts[:, :500])
    for k in ("code", "elem", "rst", "dist2"):
        np.testing.assert_array_equal(one[k], allc[k])
