"""bench.py keeps its contract: one JSON line with the required keys, on a
small copy of the training workload, with the digest checks passing."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_training_line_contract():
    line = run("--scale", "0.01", "--steps", "2", "--warmup", "3", "--serving-window", "2")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] > 0 and line["gpu_launches"] > 0
    assert line["verified"]["cow_image_equals_memory_at_t1"]
    assert line["verified"]["recopy_image_equals_memory_at_t2"]
    assert line["verified"]["iterative_recopy_image_equals_memory_at_t2"]
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r
    assert line["cpu_baseline"]["kind"] == "oracle"
    rows = {r["kernel"].split(",")[0]: r for r in line["rooflines"][1:]}
    assert rows["k_validate_rounds"]["frac"] > 0
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert "all_cores" in line["cpu_baseline"]["loops"]
    # the batched, serving and restore forms, measured in the same run
    arms = line["arms"]
    assert set(arms) == {"batched", "serving", "restore"}
    for name, arm in arms.items():
        assert "error" not in arm, (name, arm)
        assert arm["value"] > 0 and arm["gpu_launches"] > 0 and "clocks" in arm
    assert arms["batched"]["status"] == 0 and "roofline" in arms["batched"]
    assert arms["serving"]["p99_ms"] > 0 and "one_at_a_time" in arms["serving"]
    assert arms["restore"]["verified"]["final_memory_equals_stw_restore_plus_replay"]


def test_reference_arm_contract():
    line = run("--impl", "reference", "--steps", "1", "--warmup", "1")
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
