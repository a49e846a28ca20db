"""bench.py's output contract, on the host.

The reference arm (the oracle on the host cores, one maneuver layer of the
512^3 parking workload per step) prints one JSON line with the metric, the
unit, the workload, a cpu_baseline describing the run and an e2e object with
no host-device copies.  The library's own arm needs a GPU: without one it
ends with an error instead of falling back to the CPU.
"""
import json
import os
import subprocess
import sys

from tests.util import ROOT


def _run(args, timeout):
    env = dict(os.environ, PYTHONPATH=ROOT, CUDA_VISIBLE_DEVICES="")
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = _run(["--impl", "reference", "--steps", "1", "--warmup", "3"], timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "pose-cell updates/s" and d["unit"] == "updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["config"]["workload"] == "parallel_parking_512x512x512_N8"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_library_arm_fails_without_a_gpu():
    r = _run(["--steps", "1", "--warmup", "3", "--no-served", "--no-batched", "--no-maze"], timeout=300)
    assert r.returncode != 0
    assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")], "no result line without a GPU"
