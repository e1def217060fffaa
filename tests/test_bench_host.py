"""Host logic of bench.py that needs no GPU: the clock-sample summary that
goes into the bench line (median SM clock, throttle reasons seen)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_clock_summary_median_and_reasons(tmp_path):
    import bench
    path = tmp_path / "clocks.csv"
    # index, sm, sm max, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    rows = ["0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1100.2, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line"]
    path.write_text("\n".join(rows) + "\n")
    clk = bench.ClockSampler("0", str(path))
    s = clk.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["power_w_max"] == 1400.0


def test_clock_summary_without_samples(tmp_path):
    import bench
    clk = bench.ClockSampler("0", str(tmp_path / "missing.csv"))
    s = clk.summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["unsampled"] and s["samples"] == 0


def test_clock_samples_default_to_a_temporary_file():
    import tempfile

    import bench
    clk = bench.ClockSampler("0")
    assert os.path.dirname(clk.path) == tempfile.gettempdir()
