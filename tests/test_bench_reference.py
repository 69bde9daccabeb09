"""bench.py's reference arm (the oracle timed on the host cores) runs without a
GPU and prints the benchmark's JSON line with its own timing as the
cpu_baseline and e2e values; with the default (autotuned) tile it takes the
tile the autotuner picks on this workload."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "Mpixel/s" and d["higher_is_better"] is True
    assert "tile 8" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
