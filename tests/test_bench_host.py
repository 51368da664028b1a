"""Host logic of bench.py that needs no GPU: the clock record keeps only the
samples taken inside the timed region."""
import datetime

import bench


class _FakeSmi:
    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def _line(ts, sm, reasons=("Not Active",) * 4, power=900.0):
    stamp = datetime.datetime.fromtimestamp(ts).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    return ", ".join([stamp, "0", str(sm), "2070", str(power), "0x0"] + list(reasons))


def test_clock_samples_outside_the_timed_region_are_dropped():
    t0 = 1_800_000_000.0
    rows = [_line(t0 - 0.2, 2070), _line(t0 - 0.1, 2070)]                  # idle lead-in
    rows += [_line(t0 + 0.01 + 0.025 * k, 1800 + k) for k in range(5)]     # under load
    rows += [_line(t0 + 0.5, 2070, ("Active", "Not Active", "Not Active", "Not Active"))]   # after
    c = bench.ClockSampler(0, enabled=False)
    c.p = _FakeSmi("\n".join(rows) + "\n")
    r = c.stop(t0, t0 + 0.2)
    assert r["samples"] == 5 and r["in_timed_region"]
    assert r["sm_mhz"] == 1802.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == []                      # the hw_slowdown sample came after the region


def test_clock_region_shorter_than_the_period_takes_the_nearest_samples():
    t0 = 1_800_000_000.0
    rows = [_line(t0 - 0.3, 2070), _line(t0 + 0.031, 1500), _line(t0 + 0.9, 2070,
                                                                   ("Not Active",) * 3 + ("Active",))]
    c = bench.ClockSampler(0, enabled=False)
    c.p = _FakeSmi("\n".join(rows))
    r = c.stop(t0, t0 + 0.02)
    assert not r["in_timed_region"] and r["samples"] == 2
    assert r["sm_mhz"] == (1500 + 2070) / 2


def test_clock_record_without_nvidia_smi_is_none():
    assert bench.ClockSampler(0, enabled=False).stop(0.0, 1.0) is None


def test_reference_arm_prints_one_valid_line():
    """bench.py --impl reference times the oracle on the host cores and prints
    the contract's JSON line (no GPU needed)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--n", "300000"], capture_output=True, text=True, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "steps/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "matern52_n4m"
    # the reference arm times the whole series, the configuration the GPU arm runs
    assert d["config"]["n"] == 300000 and "sample_steps" not in d["config"]
    assert abs(d["ms_per_step"] - 1e3 * 300000 / d["value"]) <= 1e-9 * d["ms_per_step"]
