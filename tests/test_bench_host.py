"""CPU checks of bench.py's host logic: the reference arm (the FP64 oracle on
host cores) prints one JSON line with the contract's keys from rank 0 and
nothing from other ranks; the clock record is read from nvidia-smi's lines."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          capture_output=True, text=True, env=env, cwd=ROOT, timeout=600)


def test_reference_arm_prints_one_contract_line():
    out = run_bench({"RANK": "0", "WORLD_SIZE": "1"}, "--steps", "1", "--warmup", "0")
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    assert rec["value"] > 0 and rec["higher_is_better"] is True
    assert rec["steps"] == 1 and rec["warmup"] == 0
    assert rec["unit"] == rec["e2e"]["unit"] and rec["e2e"]["value"] == rec["value"]
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["d2h_bytes_per_step"] == 0
    cb = rec["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == rec["value"]
    assert "workload" in rec["config"]


def test_reference_arm_other_ranks_exit_without_work():
    out = run_bench({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "0")
    assert out.returncode == 0
    assert out.stdout.strip() == ""


def test_clock_summary_reads_nvidia_smi_lines():
    import bench
    clk = bench.ClockSampler(0)
    clk.lines = [
        "1965, 2070, 812.4, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 640.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "2025, 2070, 700.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
        "garbled",
    ]
    s = clk.summary()
    assert s == {"sm_mhz": 2025.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    clk.lines[1] = "1200, 2070, 640.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    assert clk.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    clk.lines = []
    assert clk.summary()["sm_mhz"] is None
