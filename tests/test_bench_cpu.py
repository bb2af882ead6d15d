"""bench.py's reference arm on the CPU: one JSON line with the contract's keys (the FP64 oracle
timed on this host), and nothing from ranks other than 0."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

KEYS = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _run(env_extra):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", **env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    lines = _run({})
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["unit"] == "evals/s" and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("tiny")


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_reference_arm_timed_steps_fit_the_run():
    """ms_per_step is the measured time of one step (one oracle run of the sample), so the
    steps' total fits inside the process's own wall time."""
    import time

    t0 = time.perf_counter()
    d = json.loads(_run({})[0])
    wall = time.perf_counter() - t0
    assert d["steps"] * d["ms_per_step"] / 1e3 <= wall


def test_calibration_sample_is_one_wavelength_exposure_slice():
    """The million-parameter calibration is sampled as one (wavelength, exposure) slice of its
    128 PSFs at full size; the binary-star evaluation is taken whole."""
    sys.path.insert(0, ROOT)
    import bench

    sub, data, frac, desc, start = bench.oracle_sample("calib")
    assert start.n_psf == 128 and sub.n_psf == 1 and frac == 1.0 / 128
    assert sub.n_pupil == 512 and sub.n_det * sub.oversample == 2048 and data.shape == (1, 1024, 1024)
    assert "slice" in desc
    cfg = bench.workload_config("calib", start, False, 1)
    assert (cfg["psfs_per_eval"], cfg["pupil"], cfg["mft_out"]) == (128, 512, 2048)
    assert cfg["l2"].startswith("no flush")
    _, _, frac_b, _, start_b = bench.oracle_sample("binary")
    assert frac_b == 1.0 and start_b.n_psf == 64
