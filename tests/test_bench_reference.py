"""The benchmark's reference arm (the CPU oracle, timed) prints one JSON line
with the contract's keys, on the CPU alone."""
import json
import os
import subprocess
import sys

from conftest import ROOT

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(*args):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_sweep_reference_line():
    d = _run("--steps", "1", "--warmup", "1", "--cpu-sample", "4")
    assert KEYS <= set(d) and d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_truncated_reference_line():
    d = _run("--workload", "truncated", "--tz-replicates", "500", "--steps", "1", "--warmup", "1")
    assert KEYS <= set(d) and d["unit"] == "replicates/s" and d["value"] > 0
    assert d["config"]["replicates_per_step"] == 900 * 500
