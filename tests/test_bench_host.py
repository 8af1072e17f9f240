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
    """Algorithmic work per located point at N=7 (n = 8): FP64 form seed + K
    iterations on the FP64 pipe; mixed form seed + K iterations in FP32 and
    the final FP64-accuracy step; no refinement steps counted."""
    n = 8
    assert bench.SEED == pytest.approx(n ** 3 * 8, rel=0.01)                 # 3 sub, 3 mul, 2 add per node
    assert bench.ITER == pytest.approx(2 * (6 * n ** 3 + 9 * n ** 2 + 12 * n) + 6 * n ** 2 * 2, rel=0.02)
    assert bench.FINAL == pytest.approx(2 * 3 * (n ** 3 + n ** 2 + n) + 0.3e3, rel=0.01)
    assert bench.EVAL1 == pytest.approx(2 * (n ** 3 + n ** 2 + n), rel=0.01)
    assert bench.WORK["fp64"] == {"f64": pytest.approx(4.1e3 + 3.43 * 8.4e3), "f32": 0.0, "f64acc": 0.0}
    assert bench.WORK["mixed"] == {"f64": 0.0, "f32": pytest.approx(4.1e3 + 3.43 * 8.4e3), "f64acc": 3.8e3}


def test_roofline_fraction_recomputes_from_its_parts():
    """frac = algorithmic work x units / kernel time / measured peak, for
    both forms; the step fraction adds the eval's work; the FP64 view puts
    the whole step's work on the FP64 pipe."""
    peaks = {"p64": 1.2, "p32": 70.0, "pdf": 6.0, "clocks": {"sm_mhz": 2070.0}}
    P, F = 10_000_000, 5
    for form in ("fp64", "mixed"):
        km = {"newton": 40.0 if form == "mixed" else 300.0}
        r = bench.roofline_form(form, P, F, km, 60.0 if form == "mixed" else 350.0, peaks, 6789.6, 1.0e7,
                                4.0e8, 6.7e8)
        w = bench.WORK[form]
        if form == "fp64":
            t = P * w["f64"] / 1.2e12
            assert r["achieved"] == pytest.approx(P * w["f64"] / 0.300 / 1e12)
            te = P * F * bench.EVAL1 / 1.2e12
        else:
            t = P * (w["f32"] / 70e12 + w["f64acc"] / 6e12)
            te = P * F * bench.EVAL1 / 6e12
        assert r["frac"] == pytest.approx(t / (km["newton"] / 1e3))
        assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
        step_ms = 60.0 if form == "mixed" else 350.0
        assert r["step"]["frac"] == pytest.approx((t + te) / (step_ms / 1e3))
        fp64 = P * (bench.SEED + bench.K_ORACLE * bench.ITER + F * bench.EVAL1) / 1.2e12
        assert r["fp64_roofline"]["frac"] == pytest.approx(fp64 / (step_ms / 1e3))


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
