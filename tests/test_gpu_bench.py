"""GPU: bench.py's own arm prints one JSON line with the contract's keys on a small workload
(the tiny configuration, a few steps): throughput, the roofline of the dominant kernel, the
end-to-end figure through host buffers, the launch count and the sampled clocks."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"}


def test_bench_line_contract():
    r = subprocess.run([sys.executable, "bench.py", "--workload", "tiny", "--steps", "5", "--warmup", "3",
                        "--no-forms", "--no-cpu"], cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["n_gpus"] == 1 and d["steps"] == 5 and d["warmup"] == 3 and d["value"] > 0
    assert d["ms_per_step"] == pytest.approx(1e3 / d["value"], rel=1e-6)
    assert d["scaling"] == "weak" and d["higher_is_better"] is True and d["data"] == "synthetic"
    ro = d["roofline"]
    assert ro["bound"] == "tensor" and ro["unit"] == "TFLOP/s" and ro["peak"] > 0
    assert ro["frac"] == pytest.approx(ro["achieved"] / ro["peak"], rel=1e-6)
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= 5 * 8  # at least eight kernels per evaluation
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    assert d["config"]["workload"].startswith("tiny")
