"""The reference arm of bench.py (the oracle on the host cores) prints the one JSON line of
the benchmark contract, for the single-LP workloads and for the batch (CPU only: small
samples)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(*args):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("args", [("--workload", "tiny"), ("--workload", "medium", "--scale", "0.01"),
                                  ("--workload", "qap", "--qap-n", "5")])
def test_reference_line(args):
    d = _run(*args, "--steps", "2", "--warmup", "1", "--sample-iters", "30")
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["unit"] == "iter/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert isinstance(d["config"]["workload"], str) and d["config"]["workload"]


def test_reference_line_batch():
    d = _run("--workload", "batch", "--count", "3", "--scale", "0.02", "--max-iter", "300",
             "--steps", "1", "--warmup", "0")
    assert KEYS <= set(d)
    assert d["impl"] == "reference" and d["unit"] == "iter/s" and d["value"] > 0
    assert d["metric"].startswith("HPR iterations/s summed over the LPs")
