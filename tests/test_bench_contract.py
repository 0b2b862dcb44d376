"""Host-side checks of the benchmark (no GPU).  The reference arm
(`bench.py --impl reference`) times the CPU oracle on bounded samples of a
workload and prints one JSON line with the keys every bench line carries;
under a multi-rank launch only rank 0 runs and prints.  It runs here on the
smallest workload (20,000 x 128, one list), in a few seconds.  The roofline's
DRAM-traffic table is keyed so that the default line finds its figure."""
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


def test_dram_traffic_figure_is_keyed_by_the_default_workload():
    """The bench line's roofline traffic comes from a table keyed by the full
    workload description, so a resized run reports none; the default run's
    workload (the 10M x 768 BF16 IVF line) must find its figure."""
    import argparse
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(config=3, n=0, queries=0, nlist=0)
    name = bench.workload_name(bench.workload_spec(args))
    assert name in bench.TRAFFIC, name
    assert 1e9 < bench.TRAFFIC[name] < 1e11
    resized = bench.workload_name(bench.workload_spec(argparse.Namespace(
        config=3, n=500_000, queries=2000, nlist=256)))
    assert resized not in bench.TRAFFIC
