"""The benchmark's JSON line on a GPU, on the tiny box: the keys the
measurement contract asks for (device time, end to end through the C ABI
with host buffers, roofline with its peak, launch count, clocks, CPU
baseline), and the DEM-only mode's line."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args):
    out = subprocess.run([sys.executable, "bench.py", "--workload", "tiny", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=900, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_bench_line_has_the_contract_keys():
    d = _bench("--steps", "3", "--warmup", "3", "--no-variants")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline", "phases"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["gpu_launches"] > 0
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["peak"] > 0 and r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    # end to end includes the host copies: not faster than the device-timed step
    assert e["ms_per_step"] >= 0.5 * d["ms_per_step"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert {"interp", "spread", "dem_contacts", "dem_update"} <= set(d["phases"])


def test_dem_only_line():
    d = _bench("--dem-only", "--steps", "2", "--warmup", "1")
    assert d["metric"].startswith("particle-steps/s (DEM sub-steps only")
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert {"dem_contacts", "dem_update"} <= set(d["phases"])
    assert d["phases"]["dem_contacts"]["launches_per_step"] == 50
