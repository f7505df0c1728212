"""CPU checks of bench.py's reference arm (the FP64 oracle on host cores):
one JSON line with the contract's keys from rank 0, nothing from other ranks."""
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
