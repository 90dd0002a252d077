"""The benchmark's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the keys of the benchmark contract; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "impl", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference"
    assert line["unit"] == "projections/s" and line["value"] > 0
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["dtype"] == "f64" and "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == line["value"] and cb["unit"] == line["unit"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # a step is one iteration on a band of rows; value scales it to whole 2048^2
    # projections of 50 iterations: value = (band pixels / 2048^2) / (50 step times)
    rows = int(cb["sample"].split("(")[1].split("x")[0])
    expect = (rows * 2048 / 2048 ** 2) / (50 * line["ms_per_step"] / 1e3)
    assert abs(line["value"] / expect - 1.0) < 1e-2


def test_reference_arm_config_is_the_gpu_arms():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2601_22793_gb300 import phantoms as ph
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    wl, _ = ph.ellipsoids_mono(seed=bench.PHANTOM_SEED)
    assert line["config"] == json.loads(json.dumps(bench.bench_config(wl, 1)))


def test_cpu_baseline_leg_times_one_and_all_cores_and_returns_the_data():
    sys.path.insert(0, ROOT)
    import bench
    rec, D = bench.cpu_baseline(1)
    assert rec["kind"] == "oracle" and rec["cores"] == (os.cpu_count() or 1)
    assert rec["value"] > 0 and rec["single_thread"]["value"] > 0 and rec["cpu_model"]
    assert D.shape == (2048, 2048) and D.dtype.name == "float32"
    oc = rec["other_configs"]   # the other configurations' oracle timings
    assert oc["spheres_mono_256"]["projections_per_s"] > 0
    assert oc["ellipsoids_poly_2048x8"]["s_per_iteration"] > 0
    assert oc["uneven_4line"]["equiv_2048sq_iterations_per_s"] > 0
    # the reference arm solves the same data
    _, _, _, D2 = bench._oracle_workload()
    assert (D == D2).all()
