"""The bench's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract the GPU arm keeps: one line, the same metric, unit and
config as our arm for the same flags, the oracle described in cpu_baseline,
an e2e object without device copies; under torchrun only rank 0 prints.
Runs on CPU: the reference arm touches no GPU."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=e,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    lines = run_bench(["--impl", "reference", "--steps", "2", "--warmup", "1", "--n", "8192"])
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["value"] > 0
    assert d["ms_per_step"] == pytest.approx(1e3 * 8192 / d["value"], rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the same config our arm reports for the same flags
    old = sys.argv
    try:
        sys.argv = ["bench.py", "--n", "8192"]
        a = bench.parse()
    finally:
        sys.argv = old
    assert d["config"] == bench.config(a, 1)
    assert d["config"]["n"] == 8192 and "workload" in d["config"]


def test_reference_arm_other_ranks_are_silent():
    lines = run_bench(["--impl", "reference", "--steps", "1", "--warmup", "0", "--n", "4096"],
                      env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert lines == []


def test_kernels_per_step_composition():
    """Launches of one plain step: reset, kick+drift+bbox, domains, keys, 8
    sort passes, reorder, 4 build launches, the two multipole passes, walk,
    kick (21), a second walk instantiation for groups that may exceed 16
    bodies, 2 launches of sibling packing (24 in the ncu launch list of the
    bench workload)."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.kernels_per_step(16, 0) == 21
    assert bench.kernels_per_step(32, 0) == 22
    assert bench.kernels_per_step(32, 1) == 24
    assert bench.kernels_per_step(64, 1) == 24
