"""bench.py's one JSON line: the oracle's reference arm on the host cores, and the B300 arm
(needs a GPU).  Checks the keys and units the benchmark contract fixes, not the numbers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
             "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "e2e"}


def _line(args, timeout):
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT,
                       capture_output=True, text=True, timeout=timeout)
    assert p.returncode == 0, p.stderr[-3000:]
    lines = [s for s in p.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1, p.stdout[-3000:]
    return json.loads(lines[0])


def test_reference_arm_prints_the_contract_line():
    d = _line(["--impl", "reference", "--workload", "nav256_d3", "--steps", "2", "--warmup", "1"],
              600)
    assert BASE_KEYS <= d.keys()
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "particle-steps/s"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1 and d["higher_is_better"]
    assert d["config"]["workload"].startswith("nav2d N=256 D=3")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


@pytest.mark.gpu
def test_vopp_arm_prints_the_contract_line():
    d = _line(["--steps", "3", "--warmup", "3", "--no-cpu-baseline", "--no-batch-serve"], 900)
    assert BASE_KEYS <= d.keys()
    assert d["value"] > 0 and d["unit"] == "particle-steps/s" and d["n_gpus"] == 1
    assert d["steps"] == 3 and d["warmup"] == 3 and d["scaling"] in ("weak", "strong")
    assert d["config"]["workload"].startswith("nav2d N=1024 D=4") and "l2" in d["config"]
    r = d["roofline"]
    assert r["bound"] in ("hbm", "tensor", "alu") and r["achieved"] > 0 and r["peak"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-6 and 0.0 < r["frac"] < 1.5
    assert "traffic" in r and r["unit"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0
    c = d["clocks"]
    assert c is None or (c["sm_max_mhz"] > 0 and isinstance(c["reasons"], list))
