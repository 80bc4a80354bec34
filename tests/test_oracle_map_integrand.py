"""Pins for the oracle's grid map and integrands (CPU only).

The map is pinned against calculus (identity on a uniform grid, unit mean
Jacobian, change-of-variables quadrature); the integrands against their
closed-form integrals computed with scipy quadrature and erf/atan.
"""
import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

import oracle
from paper_2002_12921_b300 import workloads as W

TWO32 = 2.0 ** 32


@pytest.mark.parametrize("nbins", [1, 2, 7, 50, 100, 1000])
def test_uniform_grid_map_is_identity(nbins):
    """On e_l = l/N the map is x = (w + 1/(2N)) 2^-32 and J = 1 (plain MC)."""
    rng = np.random.default_rng(nbins)
    w = rng.integers(0, 2**32, size=(20000, 3), dtype=np.uint64).astype(np.uint32)
    w[:6, 0] = [0, 1, 2**31, 2**32 - 2, 2**32 - 1, 12345]
    x, J, bins = oracle.map_samples(oracle.uniform_grid(3, nbins), w)
    y = (w.astype(np.float64) + 0.5 / nbins) / TWO32
    assert np.allclose(x, y, rtol=0, atol=4e-16)
    # Delta_j = (j+1)/N - j/N carries a rounding error of up to one ulp of 1,
    # i.e. a relative error of N eps per dimension
    assert np.all(np.abs(J - 1.0) <= 3 * 2 * nbins * np.finfo(float).eps)
    assert np.array_equal(bins, (w.astype(np.uint64) * nbins >> 32).astype(np.int32))
    assert bins.min() >= 0 and bins.max() <= nbins - 1


def test_map_monotone_continuous_and_hits_edges():
    """x(w) is non-decreasing; the first word of bin j maps to e_j."""
    N = 37
    e = W.random_monotone_grid(1, N, seed=5, spread=1.5)
    w = np.sort(np.random.default_rng(0).integers(0, 2**32, 100000, dtype=np.uint64))
    x, _, _ = oracle.map_samples(e, w.astype(np.uint32).reshape(-1, 1))
    assert np.all(np.diff(x[:, 0]) >= 0)
    first = np.ceil(np.arange(N) * TWO32 / N).astype(np.uint64).astype(np.uint32)
    xs, _, b = oracle.map_samples(e, first.reshape(-1, 1))
    assert np.array_equal(b[:, 0], np.arange(N))
    width = np.diff(e[0])
    assert np.all(np.abs(xs[:, 0] - e[0, :-1]) <= width * N / TWO32 * 2 + 1e-16)


@pytest.mark.parametrize("nbins", [3, 50])
def test_mean_jacobian_is_one(nbins):
    """With M words evenly spread over [0, 2^32) (M a multiple of N) every bin
    gets M/N of them, so mean J = sum_j Delta_j = 1: a dropped factor N or a
    wrong width fails this."""
    e = W.random_monotone_grid(2, nbins, seed=nbins, spread=2.0)
    M = nbins * 4096
    w = np.floor((np.arange(M) + 0.5) * TWO32 / M).astype(np.uint64).astype(np.uint32)
    _, J, _ = oracle.map_samples(e[:1], w.reshape(-1, 1))
    assert abs(J.mean() - 1.0) < 1e-12


def test_change_of_variables_midpoint_rule():
    """mean over evenly spread words of f(x(y)) J(y) -> int_0^1 f(x) dx (midpoint
    rule in y on a non-uniform grid), for f = x^2 and f = cos(3x)."""
    N = 20
    e = W.random_monotone_grid(1, N, seed=11, spread=1.0)
    M = N * 20000
    w = np.floor((np.arange(M) + 0.5) * TWO32 / M).astype(np.uint64).astype(np.uint32)
    x, J, _ = oracle.map_samples(e, w.reshape(-1, 1))
    assert abs(np.mean(x[:, 0] ** 2 * J) - 1.0 / 3.0) < 1e-8
    assert abs(np.mean(np.cos(3 * x[:, 0]) * J) - np.sin(3.0) / 3.0) < 1e-8


def gauss_closed(a, mu):
    mu = np.asarray(mu, dtype=np.float64)
    return float(np.prod(0.5 * (erf((1 - mu) / a) + erf(mu / a))))


@pytest.mark.parametrize("a,mu", [(0.1, 0.5), (0.15, 0.33), (0.3, 0.8)])
def test_gauss_integrand_normalisation_1d(a, mu):
    """Eq. 1 with N = (a sqrt(pi))^-d: int_0^1 = (erf((1-mu)/a) + erf(mu/a))/2."""
    p = W.gauss_params(1, a, mu)
    val, _ = integrate.quad(lambda t: oracle.integrand(W.GAUSS, p, np.array([[t]]))[0], 0, 1,
                            points=[mu], epsabs=1e-13, epsrel=1e-12, limit=200)
    assert abs(val - gauss_closed(a, [mu])) < 1e-10
    peak = oracle.integrand(W.GAUSS, p, np.array([[mu]]))[0]
    assert abs(peak - 1.0 / (a * np.sqrt(np.pi))) < 1e-12 * peak


def test_gauss_integrand_2d_and_mixture():
    a = 0.2
    p = W.gauss_params(2, a, [0.4, 0.6])
    val, _ = integrate.dblquad(lambda y, x: oracle.integrand(W.GAUSS, p, np.array([[x, y]]))[0],
                               0, 1, 0, 1, epsabs=1e-12, epsrel=1e-11)
    assert abs(val - gauss_closed(a, [0.4, 0.6])) < 1e-9
    pm = W.mix2_params(2, a)
    valm, _ = integrate.dblquad(lambda y, x: oracle.integrand(W.GAUSS_MIX2, pm,
                                                              np.array([[x, y]]))[0],
                                0, 1, 0, 1, epsabs=1e-12, epsrel=1e-11)
    expect = 0.5 * (gauss_closed(a, [1 / 3, 1 / 3]) + gauss_closed(a, [2 / 3, 2 / 3]))
    assert abs(valm - expect) < 1e-9


def test_mixture_with_asymmetric_centres_by_quadrature():
    """Centres whose components differ (the symmetric (1/3, 2/3) pair above
    would not tell the two centres' coordinates apart): the quadrature of the
    mixture equals the mean of the two erf closed forms."""
    a, mu_a, mu_b = 0.15, [0.2, 0.7], [0.6, 0.35]
    p = [a] + mu_a + mu_b
    val, _ = integrate.dblquad(lambda y, x: oracle.integrand(W.GAUSS_MIX2, p,
                                                             np.array([[x, y]]))[0],
                               0, 1, 0, 1, epsabs=1e-12, epsrel=1e-11)
    expect = 0.5 * (gauss_closed(a, mu_a) + gauss_closed(a, mu_b))
    assert abs(val - expect) < 1e-9


@pytest.mark.parametrize("kind", [W.GENZ_DISC, W.GENZ_PPEAK])
@pytest.mark.parametrize("dim", [1, 2])
def test_genz_integrands_integrate_to_one(kind, dim):
    """Sec. 3.1: the factor N makes each toy integrand integrate exactly to 1."""
    p = W.genz_params(dim, seed=7 + dim, kind=kind)
    a = p[:dim]
    f = lambda *xs: oracle.integrand(kind, p, np.array([xs[::-1]]))[0]  # noqa: E731
    if dim == 1:
        val, _ = integrate.quad(lambda t: f(t), 0, 1, points=[a[0]], epsabs=1e-12, limit=200)
    else:
        opts = {"epsabs": 1e-11, "epsrel": 1e-10, "limit": 200}
        lo = [a[0], a[1]] if kind == W.GENZ_DISC else [0, 0]
        val, _ = integrate.nquad(lambda y, x: f(y, x), [[lo[1], 1], [lo[0], 1]], opts=opts)
    assert abs(val - 1.0) < 1e-8


def test_genz_disc_is_zero_below_thresholds():
    p = W.genz_params(3, seed=1, kind=W.GENZ_DISC)
    a = np.array(p[:3])
    x = np.array([[a[0] - 1e-3, 0.9, 0.9], [0.9, a[1], 0.9], [0.95, 0.95, 0.95]])
    f = oracle.integrand(W.GENZ_DISC, p, x)
    assert f[0] == 0.0 and f[1] == 0.0 and f[2] > 0.0


def test_flat_integrand():
    x = np.random.default_rng(0).random((10, 5))
    assert np.all(oracle.integrand(W.FLAT, [], x) == 1.0)
