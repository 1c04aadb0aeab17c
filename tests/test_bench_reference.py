"""bench.py's reference arm (the FP64 oracle on host cores) prints the contract's JSON
line on the same workload config as the GPU arm; no GPU needed."""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == "within-cutoff pair interactions/sec" and line["unit"] == "pairs/s"
    assert line["value"] > 0 and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    sys.path.insert(0, ROOT)
    import bench
    from paper_1611_04474_gb300 import workloads as W

    args = argparse.Namespace(mode="f32", algo=0, dt=1.0)
    expected = bench.bench_config(W.workload_lattice_92k(), args, 1)
    assert line["config"]["workload"] == expected["workload"]
    assert set(line["config"]) == set(expected)
