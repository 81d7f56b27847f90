"""The benchmark's JSON line on the CPU: the reference arm (the FP64 oracle
timed on the host cores) prints one line with every key of the contract,
and a warm-up below 3 steps is raised to 3.  The GPU arm prints the same
keys plus roofline, clocks and launches; it runs in the GPU tests' box."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"),
                          *args], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    d = _run("--impl", "reference", "--steps", "2", "--warmup", "1")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC
    assert d["unit"] == "GLUPS" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2
    assert d["warmup"] == 3  # raised to the minimum
    assert d["vs_baseline"] is None
    assert d["scaling"] == "weak" and d["data"] == "synthetic"
    assert d["dtype"] == "f64"
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


@pytest.mark.gpu
def test_gpu_arm_line_small_batch():
    d = _run("--lattices", "4", "--steps", "3", "--warmup", "3",
             "--e2e-steps", "3", "--compare", "fp32")
    assert "impl" not in d or d["impl"] != "reference"
    assert d["value"] > 0 and d["unit"] == "GLUPS"
    assert d["steps"] == 3 and d["warmup"] == 3
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    # achieved counts the algorithmic bytes (16-bit storage: 89 B per fluid
    # node plus 16 B per surface node), not the layout's own
    assert 89.0 <= r["bytes_per_fluid_node"] < 89.0 + 16.0
    assert r["stored_bytes_per_fluid_node"] >= r["bytes_per_fluid_node"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0
    assert e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 3
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    assert d["compare"]["precision"] == "fp32"
    assert d["compare"]["glups_per_gpu"] > 0
