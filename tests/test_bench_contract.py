"""The benchmark's command-line contract, on the host (no GPU).

The reference arm times the FP64 oracle on the host cores and prints one JSON line with
the metric, unit and direction of the GPU arm, a cpu_baseline object describing the run
and an e2e object with no host<->device bytes.  The GPU arm on a machine without a GPU
must fail loudly: no result line, a non-zero exit, never a silent CPU fallback.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BENCH = os.path.join(ROOT, "bench.py")

pytestmark = pytest.mark.skipif(
    __import__("torch").cuda.is_available(), reason="host-only checks (a GPU is present)")


def _run(*args, timeout=600):
    return subprocess.run([sys.executable, BENCH, *args], cwd=ROOT, capture_output=True, text=True,
                          timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--workload", "two_species_small", "--steps", "1", "--warmup", "1")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("Mparticles/s") and d["unit"] == "Mparticles/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "two_species_small"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_gpu_arm_fails_loudly_without_a_gpu():
    r = _run("--workload", "two_species_small", "--steps", "1", "--warmup", "1", "--no-extras",
             "--no-cpu-baseline", "--e2e-steps", "0")
    assert r.returncode != 0
    assert not [l for l in r.stdout.splitlines() if '"value"' in l], r.stdout
