"""The benchmark's reference arm (the oracle timed on the host cores) keeps the JSON contract:
one line with impl "reference", the metric and unit of the GPU arm, a cpu_baseline describing
the run and an e2e entry with no host-device traffic. One bounded step, no warm-up (CPU only)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "field solves/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"].startswith("field solves/s")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("cw-mixed-64x64x48")
