"""bench.py's reference arm on the host cores: the complete FP64 oracle (set-up and one
complete solve on a pool of all host cores, then a bounded sample per step), printed as one
JSON line with the fields the GPU arm prints (same metric, config and unit, `impl:
reference`, the CPU baseline it is, an e2e block with no host-device copies).  Run here on
the 8^3 channel so that it takes seconds; the benchmark size differs only in its sizes."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.slow
def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--m", "8"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [json.loads(x) for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] == d["value"] and d["steps"] == 2
    assert d["config"]["workload"].startswith("channel8_")
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert d["oracle"]["iterations"] > 0 and d["oracle"]["relres"] <= 1e-8
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
