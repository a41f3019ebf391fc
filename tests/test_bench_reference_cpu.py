"""bench.py's reference arm on the CPU: the oracle timed on the host cores prints one JSON line
with the benchmark's metric, unit and configuration, marked as the reference implementation."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_json_line():
    import __graft_entry__

    __graft_entry__.build()
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["higher_is_better"] is True
    assert out["metric"].startswith("grid-pt RK-stage updates/s")
    assert out["unit"] == "grid-pt RK-stage updates/s" and out["value"] > 0
    assert out["config"]["workload"] == "sbli-2048x384x256"
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
    assert (out["steps"], out["warmup"], out["n_gpus"]) == (1, 3, 1)
