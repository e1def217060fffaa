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


def _reference_arm(env_extra):
    import json
    import subprocess
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--ref-n", "32"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference times the CPU oracle and prints one JSON line
    with the keys of the bench contract, on the host (no GPU needed)."""
    (line,) = _reference_arm({"RANK": "0", "WORLD_SIZE": "1"})
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["unit"] == "Mpoint-steps/s" and line["higher_is_better"]
    assert line["dtype"] == "f64" and line["data"] == "synthetic" and line["vs_baseline"] is None
    assert abs(line["ms_per_step"] * line["value"] - 32 * 32 * 1e-3) < 1e-6 * 32 * 32
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert "32x32" in cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in line["config"]


def test_reference_arm_is_silent_on_other_ranks():
    assert _reference_arm({"RANK": "1", "WORLD_SIZE": "2"}) == []
