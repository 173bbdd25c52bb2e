"""Host-side logic of bench.py (no GPU): the byte counts behind the bench
line's value and roofline, and the clock sampler's summary of nvidia-smi
readings (median SM clock, throttle reasons, the timed-region window)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_host", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_sweep_bytes_of_the_benchmark_solve(bench):
    # X once per sweep (4 bytes x 1,000,000 x 256) plus the read and write of e (8m)
    assert bench.sweep_bytes(1_000_000, 256, 4, 5) == 5 * (4 * 256 + 8) * 1_000_000
    assert bench.sweep_bytes(1_000_000, 256, 4, 5) == 5_160_000_000
    # e kept on chip (the wide and batched kernels): X alone
    assert bench.sweep_bytes(2000, 200_000, 4, 2, e_in_hbm=False) == 2 * 4 * 2000 * 200_000


def test_solve_bytes_add_the_setup_read(bench):
    m, n = 4_000_000, 512
    for esz in (2, 4):
        for sweeps in (1, 4, 9):
            setup = esz * m * n + 4 * m  # one read of X (Gram, X^T y) and of y
            assert bench.setup_bytes(m, n, esz) == setup
            assert bench.solve_bytes(m, n, esz, sweeps) == setup + bench.sweep_bytes(m, n, esz, sweeps)


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", pcap="Not Active"):
    return f"{sm}, {mx}, 900.0, {hw}, {hwt}, {swt}, {pcap}"


def test_clock_summary_median_reasons_and_window(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [(0.00, _line(1200, 2070, hw="Active")),  # before the timed region
                (1.00, _line(2070, 2070)),
                (1.02, _line(2055, 2070, pcap="Active")),
                (1.04, _line(2070, 2070)),
                (9.00, _line(800, 2070, swt="Active"))]   # after it
    cs.mark(0.99, 1.05)
    s = cs.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3 and s["in_timed_region"]
    cs.window = None  # no window: every reading counts
    s = cs.summary()
    assert s["samples"] == 5 and set(s["reasons"]) == {"hw_slowdown", "sw_power_cap",
                                                       "sw_thermal_slowdown"}


def test_clock_summary_without_readings(bench):
    cs = bench.ClockSampler(0)
    cs.lines = [(0.0, "[N/A], [N/A]"), (0.1, "garbage")]
    assert cs.summary()["reasons"] == ["unsampled"]
