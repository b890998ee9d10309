"""The reference arm of bench.py (the CPU oracle) prints the one JSON line of
the benchmark contract, on the same workload config as the native arm."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    import bench
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["metric"] == bench.METRIC
    assert out["unit"] == "TFLOP/s" and out["higher_is_better"] is True
    assert out["n_gpus"] == 1 and out["steps"] == 1 and out["warmup"] == 0
    assert out["value"] > 0 and out["ms_per_step"] > 0
    assert out["config"] == bench.trevc_config(4096, 1)
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == out["value"] and cb["sample"]
    assert out["e2e"] == {"value": out["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}


def test_trevc_config_names_the_workload_only():
    import bench
    c = bench.trevc_config(4096, 1)
    assert c["m"] == 4096 and "n_b" not in c and c["eigenvectors"] == 4096
    assert "4096x4096" in c["workload"] and "268 MB" in c["l2"] and c["parallelism"] == "single GPU"
    assert bench.trevc_config(4096, 2)["parallelism"] == "replicas x2"
    assert "substitution_gemm" not in c
