"""Host-side logic of bench.py (no GPU): the clock-sample window and the
max-null KL summary."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, reasons=("Not Active",) * 4):
    return ["0", str(sm), "2070", "900.0", "0x0"] + list(reasons)


def test_clock_samples_restricted_to_the_timed_region():
    c = bench.ClockSampler(0)
    c.rows = [(1.0, _row(345)), (2.0, _row(2070)), (2.5, _row(2055)),
              (3.0, _row(2070, ("Not Active", "Not Active", "Not Active", "Active"))),
              (9.0, _row(400))]
    out = c.stop(1.9, 3.1)
    assert out["samples"] == 3 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    # no sample inside the region: every sample is reported, and flagged
    out = c.stop(4.0, 5.0)
    assert out["samples"] == 5 and out["window"].startswith("whole sampling")
    assert out["sm_mhz"] == 2055.0


def test_throttle_reasons_collected():
    c = bench.ClockSampler(0)
    c.rows = [(1.0, _row(1500, ("Active", "Not Active", "Active", "Not Active")))]
    out = c.stop(0.0, 2.0)
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_hist_kl():
    rng = np.random.default_rng(0)
    a = rng.normal(5.0, 0.3, 20000)
    b = rng.normal(5.0, 0.3, 20000)
    c = rng.normal(4.5, 0.2, 20000)
    assert bench.hist_kl(a, a) < 1e-3
    assert bench.hist_kl(a, b) < 0.02
    assert bench.hist_kl(a, c) > 1.0
    assert bench.hist_kl(a, c) > bench.hist_kl(a, b)
