"""The benchmark's reference arm (the CPU oracle) prints one JSON line with the
keys the benchmark contract names; run on a small cell so it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--ncell", "2",
                          "--radius", "6", "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "steps/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_roofline_traffic_is_keyed_to_the_default_workload(monkeypatch):
    """The DRAM traffic of the dominant kernel that the benchmark line reports
    is keyed to the workload name the default run produces: a renamed
    workload would silently report null."""
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    key = (bench.cfg_name(args), "fp32", "gemm_M=UK")
    assert key in bench.TRAFFIC and bench.TRAFFIC[key] > 0
    # a different workload has no capture
    monkeypatch.setattr(sys, "argv", ["bench.py", "--radius", "8"])
    assert (bench.cfg_name(bench.parse()), "fp32", "gemm_M=UK") not in bench.TRAFFIC
