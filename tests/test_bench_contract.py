"""The benchmark's contract on the CPU: the reference arm's JSON line (the
oracle timed on every host core), the algorithmic bytes per point behind the
roofline, and the committed ncu capture still matching the collide sources
(otherwise `traffic` would be reported as null)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_point():
    # populations 41 read + 41 written, plus 12 field values per point
    assert bench.algorithmic_bytes_per_point("f32") == {"step": 376, "collide": 356}
    assert bench.algorithmic_bytes_per_point("f16dev")["step"] == 212
    assert bench.algorithmic_bytes_per_point("bf16dev")["step"] == 212
    assert bench.algorithmic_bytes_per_point("f64")["step"] == 752
    # the paper's theta_R solver writes theta_T(f) from the collision as well
    assert bench.algorithmic_bytes_per_point("f32", "paper") == {"step": 376, "collide": 360}
    assert bench.algorithmic_bytes_per_point("f16dev", "paper")["collide"] == 196


def test_committed_collide_capture_matches_the_sources():
    traffic = bench.ncu_traffic("f32")
    assert traffic is not None, "the collide sources changed since profiles/ncu_collide_f32.txt"
    assert 300.0 < traffic[0] < 400.0


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "3", "--ref-n", "6"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["value"] > 0 and line["steps"] == 2 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
