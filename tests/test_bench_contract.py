"""The benchmark's JSON contract on the CPU: the reference arm (the CPU oracle
timed on the host cores) prints one line with every field the measurement
needs, and the workload description states where the inputs sit against L2."""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_one_complete_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--m", "65536", "--n", "16"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "rows/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f64" and d["data"] == "synthetic"
    assert d["config"]["workload"] == "tsqr_factor+form_q f64 m=65536 n=16 gaussian"
    cpu = d["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == d["value"] and cpu["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing(capsys):
    args = argparse.Namespace(m=65536, n=16, steps=1, warmup=0, gpus=2, leaf_rows=0, arity=0)
    assert bench.reference_arm(args, 2, 1) is None
    assert capsys.readouterr().out == ""


def test_workload_l2_note_follows_the_input_size():
    big = bench.workload_config(argparse.Namespace(m=4194304, n=64, leaf_rows=0, arity=0))
    assert big["l2"].startswith("inputs (2.1 GB) larger than L2")
    small = bench.workload_config(argparse.Namespace(m=65536, n=16, leaf_rows=0, arity=0))
    assert "fit in L2" in small["l2"]
    # FP32 storage halves the bytes: 4,194,304 x 64 x 4 B = 1.07 GB, still above L2.
    mixed = bench.workload_config(argparse.Namespace(m=4194304, n=64, leaf_rows=0, arity=0), dtype="f32")
    assert mixed["l2"].startswith("inputs (1.1 GB) larger than L2")
