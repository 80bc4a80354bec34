"""Host-side rules that need no GPU: which clock records reject bench.py's
timed window, the algorithmic counts its roofline and pipe fractions use, and
the binding's shape and length checks before it calls the library (the C calls
read exactly the counts their arguments imply)."""
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
    # the method's count: Philox 60 per call, 7 per dimension, 12 per sample
    assert bench.alg_ops_per_sample(8) == 120 + 56 + 12 == 188
    assert bench.alg_ops_per_sample(16) == 240 + 112 + 12
    # the kernel's count, round keys computed once per launch
    assert bench.kernel_ops_per_sample(8) == 167
    assert bench.SAMPLES_PER_STEP == 10 * 10_000_000 + 5 * 100_000_000


def test_binding_checks_shapes_before_calling_the_library():
    """Vegas.set_grid / set_box refuse arrays of the wrong shape in Python
    (the C calls read exactly dim x (nbins + 1) and dim pairs)."""
    import numpy as np
    import pytest

    from paper_2002_12921_b300 import binding as B

    v = B.Vegas.__new__(B.Vegas)  # no device: only the shape checks run
    v.dim, v.nbins, v.handle = 3, 10, None
    with pytest.raises(ValueError):
        v.set_grid(np.zeros((3, 10)))
    with pytest.raises(ValueError):
        v.set_box([(0.0, 1.0)] * 2)


def test_batch_binding_checks_lengths_before_calling_the_library():
    import pytest

    from paper_2002_12921_b300 import binding as B

    with pytest.raises(ValueError):  # a Gaussian in 3 dimensions takes 4 parameters
        B.vegas_batch_init([2, 3], [100, 100], 10, 1, B.VEGAS_FP64, [[0.1, 0.5, 0.5], [0.1]],
                           4, 0, 0, 0)
    with pytest.raises(ValueError):  # one box per integral
        B.vegas_batch_init([2, 3], [100, 100], 10, 1, B.VEGAS_FP64, [[], []], 4, 0, 0, 0,
                           integrand=B.VEGAS_FLAT, boxes=[[(0.0, 1.0)] * 2])
