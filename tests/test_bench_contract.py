"""The benchmark's reference arm on the host (no GPU): `bench.py --impl
reference` times the CPU oracle on bounded samples of a workload and prints
one JSON line with the keys every bench line carries; under a multi-rank
launch only rank 0 runs and prints.  Run on the smallest workload (20,000 x
128, one list) so that it takes a few seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, args=()):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.pop("LOCAL_RANK", None)
    env["CUDA_VISIBLE_DEVICES"] = ""  # the arm is the host oracle; inputs drawn on the CPU
    if extra_env:
        env.update(extra_env)
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--config", "1", "--steps", "2", "--warmup", "1", *args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_bench_line():
    lines = _run()
    assert len(lines) == 1
    b = json.loads(lines[0])
    assert b["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in b, key
    assert b["steps"] == 2 and b["warmup"] == 1 and b["n_gpus"] == 1
    assert b["value"] > 0 and b["ms_per_step"] > 0 and b["higher_is_better"] is True
    assert b["unit"] == "candidates/s" and b["scaling"] == "weak"
    assert b["config"]["workload"].startswith("plain-20k-d128")
    cb = b["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == b["value"] and cb["unit"] == b["unit"]
    e2e = b["e2e"]
    assert e2e["value"] == b["value"] and e2e["unit"] == b["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []
