"""The benchmark's reference arm (the CPU oracle) prints one JSON line with the keys both arms share,
the same metric and workload description as the GPU arm, and zero host<->device bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--workload", "square2d_64", "--ref-cores", "2", "--ref-iters", "10"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"):
        assert key in line, key
    sys.path.insert(0, ROOT)
    import bench
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC
    assert line["higher_is_better"] is True and line["value"] > 0
    assert line["config"]["workload"] == "square2d_64"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] == 2


def test_default_workload_is_the_largest_single_gpu_configuration():
    sys.path.insert(0, ROOT)
    import bench
    spec, B, cfg = bench.workload_spec("large256_192")
    assert cfg == 5 and B == 64 and spec.nx[0] == spec.ny[0] == 256 and spec.n_directions == 192
    assert spec.restart == 40 and spec.rx * spec.ry == 64
