"""The benchmark's JSON line on a GPU, on a reduced series: every key the
measurement contract asks for is there and consistent."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--n", "400000", "--steps", "5",
                        "--warmup", "3", "--no-extra", "--no-next", "--no-comparator"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["steps"] == 5 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["dtype"] == "f64"
    n = d["config"]["n"]
    assert n == 400000
    assert abs(d["value"] - n / (d["ms_per_step"] * 1e-3)) <= 1e-9 * d["value"]
    ro = d["roofline"]
    assert ro["bound"] == "alu" and ro["unit"] == "TFLOP/s" and 0.0 < ro["frac"] < 1.5
    assert abs(ro["frac"] - ro["achieved"] / ro["peak"]) <= 1e-12
    # the dense sequential method's flops (oracle/flops.py) over the whole call
    assert ro["algorithmic_flops_per_step"] == 575.0
    assert abs(ro["algorithmic_achieved"] - 575.0 * d["value"] / 1e12) <= 1e-9 * ro["algorithmic_achieved"]
    assert abs(ro["algorithmic_frac"] - ro["algorithmic_achieved"] / ro["peak"]) <= 1e-12
    assert d["gpu_launches"] == 5 * d["graph_replay"]["gpu_launches_per_replay"]
    e = d["e2e"]
    assert e["h2d_bytes_per_step"] == 16 * n + 24 and e["d2h_bytes_per_step"] == 32 and e["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
