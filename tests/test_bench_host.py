"""bench.py's host-side rules (no GPU): which clock records reject a timed
window, and the algorithmic counts its roofline and pipe fractions use."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_records_that_reject_a_window():
    ok = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    # the power cap is kept (normal on a 1.1 kW part), even with lower clocks
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1600.0, reasons=["sw_power_cap"]))
    # clocks stuck well below the maximum with no reason: a leftover lock
    assert bench.clocks_rejected(dict(ok, sm_mhz=1155.0))
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1900.0))
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["nvidia-smi unavailable"]})


def test_algorithmic_counts():
    # d=8: Philox rounds 0-1 shared (2 products), rounds 2-9 of two calls (32),
    # one bin split per dimension (8)
    assert bench.products_per_sample(8) == 42
    assert bench.products_per_sample(16) == 2 + 64 + 16
    assert bench.products_per_sample(1) == 2 + 16 + 1
    assert bench.alg_ops_per_sample(8) == 167
    assert bench.SAMPLES_PER_STEP == 10 * 10_000_000 + 5 * 100_000_000
