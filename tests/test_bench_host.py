"""CPU checks of bench.py's host logic: the reference arm (the FP64 oracle on
host cores) prints one JSON line with the contract's keys from rank 0 and
nothing from other ranks; the clock record is read from nvidia-smi's lines;
the CPU sample is scaled by the oracle's own solve counts, which are the
oracle's."""
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


def test_cpu_sample_is_scaled_by_the_oracle_solve_counts():
    """The CPU baseline scales a timed sample of oracle iterations to the
    oracle's own solve: start-up + iterations x (sweep + rest) + (f/g
    evaluations - 1) x the mean evaluation, the means taken over the sampled
    iterations after the skipped ones (a line search may take 1 or 20
    evaluations, so a per-iteration mean would be skewed)."""
    import bench
    full = bench.oracle_solve("dense_256")
    s = {"workload": "dense_256", "t_init_s": 2.0, "per_iter_s": [30.0, 5.0, 7.0],
         "sweep_s": [1.0, 1.0, 1.0], "fg_count": [20, 3, 5], "fg_s": [28.0, 3.6, 5.6]}
    e = bench.extrapolate(s, 1)
    fg = (3.6 + 5.6) / 8
    rest = ((5.0 - 1.0 - 3.6) + (7.0 - 1.0 - 5.6)) / 2
    want = 2.0 + full["iters"] * (1.0 + rest) + (full["fg_evals"] - 1) * fg
    assert abs(e["est_solve_s"] - want) <= 1e-9 * want
    assert e["oracle_iters"] == full["iters"] and e["oracle_fg_evals"] == full["fg_evals"]
    assert bench.extrapolate(dict(s, workload="no_such_workload"), 0)["est_solve_s"] is None
    assert bench.extrapolate(s, 3)["est_solve_s"] is None


def test_stored_oracle_solves_are_the_oracles_own():
    """oracle/workload_iters.json holds the oracle's own solves (written by
    oracle/workload_iters.py, which calls only the oracle and the input
    generators).  The 20^3 entry is recomputed here and must match exactly;
    every entry must be a converged solve below the tolerance."""
    import importlib.util
    import synth
    spec = importlib.util.spec_from_file_location("wi", os.path.join(ROOT, "oracle", "workload_iters.py"))
    wi = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(wi)
    stored = json.load(open(os.path.join(ROOT, "oracle", "workload_iters.json")))
    prob, u0 = synth.workload_dense_small()
    got = wi.run("dense_small", prob, u0, 3)
    for key in ("iters", "fg_evals", "restarts", "ls_failures", "converged"):
        assert got[key] == stored["dense_small"][key], key
    for key in ("f", "gnorm_over_P"):   # another host's BLAS may round differently
        assert abs(got[key] - stored["dense_small"][key]) <= 1e-10 * abs(stored["dense_small"][key]), key
    for name, rec in stored.items():
        assert rec["converged"] and rec["gnorm_over_P"] < 1e-7, name
