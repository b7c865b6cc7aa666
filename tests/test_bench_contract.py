"""The benchmark's output contract, checked without a GPU: the reference arm
(the FP64 checker timed on the host cores) prints one JSON line with the keys
the contract names, and the workload text follows the run's parameters."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_workload_text():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.workload(4096, 1, 9, 3.0, 30.0, 40, "all", 8).startswith("8 x 4096x4096 ")
    assert "box spatial W=5" in bench.workload(2048, 0, 5, 0.0, 40.0, 1, "fwd")
    assert bench.workload(2048, 0, 5, 0.0, 40.0, 1, "fwd").endswith("per image fused forward")
    assert bench.WORKLOAD == bench.workload(2048, 1, 9, 3.0, 30.0, 40, "all", 96).replace(
        "Gaussian spatial sigma_s=3 (W=9), sigma_r=30, N=40;",
        "Gaussian spatial sigma_s=3 (W=9), sigma_r=30, N=40 (bound for delta=1);")
