"""The reference arm of bench.py (the oracle timed on the host cores): its JSON line, its refusal
lines, and its behaviour on ranks other than 0.  Runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    return r.returncode, [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_line():
    rc, lines = run_bench(["--impl", "reference", "--config", "0", "--steps", "1", "--warmup", "3"])
    assert rc == 0 and len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and "sampling phase" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n"] == 900 and d["config"]["N"] == 32


def test_reference_arm_refuses_serve_and_compare():
    for cfg in ("serve", "compare"):
        rc, lines = run_bench(["--impl", "reference", "--config", cfg, "--steps", "1"])
        assert rc == 0 and len(lines) == 1
        d = json.loads(lines[0])
        assert d["impl"] == "reference" and "unavailable" in d


def test_reference_arm_runs_on_rank_zero_only():
    rc, lines = run_bench(["--impl", "reference", "--config", "0", "--steps", "1"],
                          {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert rc == 0 and lines == []
