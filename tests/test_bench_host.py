"""Host-side checks of the benchmark script (no GPU needed).

* The work model of the roofline: W(N) = 40 P(N) + 30 (N-1) + 60 (N-2)
  + 120 (N-3) + 20 N flop per replica-step with P(N) = N(N-1)/2 - (2N-3)
  nonbonded pairs; W(75) = 121 860, and 111 348 with the kernels' own
  36-flop pair count.
* More than one GPU is refused with an "unavailable" line and exit status 0.
* The reference arm (the oracle on the host cores) prints the contract's
  JSON line: the metric and unit of the GPU arm, impl "reference", a
  cpu_baseline describing the run and an e2e object without copies.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_work_model():
    assert bench.flop_per_replica_step(75) == 121860
    assert bench.flop_per_replica_step(75, bench.FLOP_PAIR_KERNEL) == 121860 - 4 * 2628
    # two atoms: one bond, no nonbonded pair
    assert bench.flop_per_replica_step(2) == 30 + 40


def _run(args, timeout=600):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return r.returncode, (json.loads(lines[-1]) if lines else None), r


def test_more_than_one_gpu_is_unavailable():
    rc, line, r = _run(["--gpus", "2", "--steps", "1", "--warmup", "3"])
    assert rc == 0, r.stderr[-2000:]
    assert "unavailable" in line and line["n_gpus"] == 2


def test_reference_arm_contract():
    rc, line, r = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    assert rc == 0, r.stderr[-2000:]
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
