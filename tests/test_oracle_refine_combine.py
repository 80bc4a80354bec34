"""Pins for the oracle's grid refinement and iteration combination (CPU only)."""
import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_2002_12921_b300 import workloads as W


# ---------------------------------------------------------------- damping
@pytest.mark.parametrize("r", [1e-12, 1e-4, 0.02, 0.3, 0.5, 0.9, 0.999999])
def test_damping_is_logarithmic_mean(r):
    """(r - 1)/ln r is the logarithmic mean of r and 1, = int_0^1 r^t dt; the
    damped weight is its alpha-th power."""
    L, _ = integrate.quad(lambda t: r ** t, 0.0, 1.0, epsabs=1e-15, epsrel=1e-13)
    assert abs(oracle.damp(r, 1.0) - L) <= 1e-12 * L
    assert abs(oracle.damp(r, 1.5) - L ** 1.5) <= 1e-12 * L ** 1.5
    assert np.sqrt(r) <= oracle.damp(r, 1.0) <= (1 + r) / 2  # GM <= LM <= AM


def test_damping_limits_and_monotone():
    assert oracle.damp(0.0, 1.5) == 0.0
    assert oracle.damp(1.0, 1.5) == 1.0
    rs = np.linspace(1e-9, 1.0, 2001)
    m = np.array([oracle.damp(r, 1.5) for r in rs])
    assert np.all(np.diff(m) > 0)


# ---------------------------------------------------------------- smoothing
def test_smoothing_linear_ramp_and_constant():
    N = 9
    ramp = np.arange(1.0, N + 1)
    s = oracle.smooth(ramp)
    assert np.allclose(s[1:-1], ramp[1:-1], rtol=1e-15)  # 3-point mean of a line
    assert s[0] == 1.5 and s[-1] == N - 0.5
    c = oracle.smooth(np.full(N, 2.5))
    assert np.all(c == 2.5)
    assert np.all(oracle.smooth(np.array([1.0, 3.0])) == 2.0)


def test_smoothing_spreads_one_hot():
    h = np.zeros(8)
    h[4] = 3.0
    assert np.allclose(oracle.smooth(h), [0, 0, 0, 1, 1, 1, 0, 0])
    h = np.zeros(8)
    h[0] = 2.0
    assert np.allclose(oracle.smooth(h), [1, 2 / 3, 0, 0, 0, 0, 0, 0])


# ---------------------------------------------------------------- refinement
def test_refine_constant_histogram_is_fixed_point():
    """P4: a flat histogram leaves any monotone grid unchanged."""
    e = W.random_monotone_grid(3, 50, seed=1, spread=1.5)
    e2 = oracle.refine(e, np.full((3, 50), 7.0), 1.5)
    # only rounding of the cumulative sums and of (target - C_b)/m_b remains
    assert np.allclose(e2, e, rtol=0, atol=1e-14)


def test_refine_scale_invariance():
    """P5: scaling a histogram row leaves the new edges unchanged (exactly for
    powers of two)."""
    e = W.random_monotone_grid(2, 30, seed=2)
    h = np.random.default_rng(3).random((2, 30)) ** 3
    base = oracle.refine(e, h, 1.5)
    assert np.array_equal(oracle.refine(e, h * 2.0 ** 70, 1.5), base)
    assert np.array_equal(oracle.refine(e, h * 2.0 ** -90, 1.5), base)
    assert np.allclose(oracle.refine(e, h * 3.7, 1.5), base, rtol=0, atol=1e-15)


def test_refine_alpha_zero_is_equal_division_of_support():
    """alpha = 0 gives weight 1 to every bin whose smoothed value is non-zero and 0
    elsewhere, so the new grid divides the support into equal shares: the inverse
    of the piecewise-linear cumulative count (numpy.interp)."""
    N = 20
    e = W.random_monotone_grid(1, N, seed=4)
    h = np.zeros((1, N))
    h[0, 8:12] = [1.0, 5.0, 2.0, 0.5]
    m = (oracle.smooth(h[0]) > 0).astype(float)
    C = np.concatenate([[0.0], np.cumsum(m)])
    expect = np.interp(np.arange(1, N) * C[-1] / N, C, e[0])
    got = oracle.refine(e, h, 0.0)
    assert np.allclose(got[0, 1:-1], expect, rtol=0, atol=1e-14)
    assert got[0, 0] == 0.0 and got[0, -1] == 1.0


@pytest.mark.parametrize("alpha", [0.5, 1.0, 1.5, 2.0])
def test_refine_against_independent_construction(alpha):
    """New edges = inverse of the cumulative damped weight, with the damping from
    its integral form and the inverse from numpy.interp."""
    N = 25
    e = W.random_monotone_grid(1, N, seed=5, spread=0.8)
    h = np.random.default_rng(6).gamma(0.7, size=(1, N))
    s = oracle.smooth(h[0])
    r = s / s.sum()
    m = np.array([integrate.quad(lambda t: ri ** t, 0, 1, epsabs=1e-15, epsrel=1e-13)[0]
                  for ri in r]) ** alpha
    C = np.concatenate([[0.0], np.cumsum(m)])
    expect = np.interp(np.arange(1, N) * C[-1] / N, C, e[0])
    got = oracle.refine(e, h, alpha)
    assert np.allclose(got[0, 1:-1], expect, rtol=0, atol=1e-12)


def test_refine_tie_at_a_zero_weight_plateau_goes_to_the_lower_bin():
    """N = 8, histogram (0, 1, 0, 0, 0, 0, 1, 0) on the uniform grid: the
    smoothed row is symmetric with zero weight in bins 3 and 4, so the
    cumulative weight equals half the total on the whole plateau [3/8, 5/8]
    and the middle target 4 (total / 8) meets it exactly.  With ties going to
    the lower bin (the reading of the re-partition rule), the middle edge is the
    plateau's lower end, 3/8; the edges stay symmetric about 1/2 otherwise."""
    e0 = np.linspace(0.0, 1.0, 9)[None, :]
    h = np.array([[0.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0, 0.0]])
    e = oracle.refine(e0, h, 1.5)[0]
    assert e[4] == 0.375
    assert np.allclose(e[1:4], 1.0 - e[7:4:-1], rtol=0, atol=1e-15)


def test_refine_one_hot_concentrates():
    """P6: all interior edges move into the hot bin and its two neighbours."""
    N = 50
    e = oracle.uniform_grid(1, N)
    h = np.zeros((1, N))
    h[0, 20] = 1.0
    got = oracle.refine(e, h, 1.5)[0]
    assert got[0] == 0.0 and got[-1] == 1.0
    assert np.all(np.diff(got) >= 0)
    assert np.all((got[1:-1] >= e[0, 19] - 1e-15) & (got[1:-1] <= e[0, 22] + 1e-15))


def test_refine_skips_zero_and_nonfinite_rows():
    e = W.random_monotone_grid(3, 10, seed=7)
    h = np.random.default_rng(1).random((3, 10))
    h[0] = 0.0
    h[2, 3] = np.inf
    got = oracle.refine(e, h, 1.5)
    assert np.array_equal(got[0], e[0]) and np.array_equal(got[2], e[2])
    assert not np.array_equal(got[1], e[1])


def test_refine_keeps_monotone_and_endpoints():
    rng = np.random.default_rng(8)
    for trial in range(20):
        N = int(rng.integers(2, 120))
        e = W.random_monotone_grid(2, N, seed=trial, spread=2.0)
        h = rng.random((2, N)) ** 6
        got = oracle.refine(e, h, 1.5)
        assert np.all(np.diff(got, axis=1) >= 0)
        assert np.all(got[:, 0] == 0.0) and np.all(got[:, -1] == 1.0)


# ---------------------------------------------------------------- combination
def test_combine_hand_examples():
    """Inverse-variance weighted mean, sigma = (sum 1/var)^-1/2, chi^2/dof."""
    m, s, c = oracle.combine([1.0, 3.0], [1.0, 1.0])
    assert (m, c) == (2.0, 2.0) and abs(s - 2 ** -0.5) < 1e-16
    m, s, c = oracle.combine([1.0, 2.0], [1.0, 4.0])  # weights 1 and 1/4
    assert abs(m - 1.2) < 1e-15 and abs(s - 1.25 ** -0.5) < 1e-15 and abs(c - 0.2) < 1e-15
    m, s, c = oracle.combine([5.0], [0.25])
    assert (m, s, c) == (5.0, 0.5, 0.0)


def test_combine_zero_variance_is_plain_mean():
    m, s, c = oracle.combine([1.0, 1.0, 1.0], [0.0, 0.0, 0.0])
    assert (m, s, c) == (1.0, 0.0, 0.0)
