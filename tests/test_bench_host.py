"""The benchmark's host side without a GPU: the CPU baseline (the FP64
oracle on one thread and on all host cores) and the reference arm's JSON
line, on the tiny box."""
import json
import os
import subprocess
import sys

import bench
from paper_2108_01814_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_cpu_baseline_records_cores():
    cb = bench.cpu_baseline(W.tiny(), 2, target=128, steps=1)
    avail, nproc = bench.host_cores()
    assert cb["kind"] == "oracle" and cb["unit"] == bench.UNIT
    assert cb["value"] > 0 and cb["single_thread"]["value"] > 0
    assert 1 <= cb["cores"] <= avail <= nproc == cb["nproc"]
    assert cb["single_thread"]["cores"] == 1
    assert f"{cb['cores']} threads" in cb["sample"]


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny",
                          "--steps", "1", "--warmup", "0", "--n-sub", "2"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
