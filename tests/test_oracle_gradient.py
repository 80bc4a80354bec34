"""Pins for the oracle's gradient of the fixed-grid Gaussian estimate (CPU)."""
import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_2002_12921_b300 import workloads as W


def closed_form(a, mu):
    """I = prod_k J_k and its exact gradient from the erf form of each factor:
    dJ/dmu = (e^{-(mu/a)^2} - e^{-((1-mu)/a)^2}) / (a sqrt(pi)),
    dJ/da = -((1-mu) e^{-((1-mu)/a)^2} + mu e^{-(mu/a)^2}) / (a^2 sqrt(pi))."""
    mu = np.asarray(mu, dtype=float)
    J = 0.5 * (erf((1 - mu) / a) + erf(mu / a))
    e0, e1 = np.exp(-(mu / a) ** 2), np.exp(-((1 - mu) / a) ** 2)
    dJmu = (e0 - e1) / (a * np.sqrt(np.pi))
    dJa = -((1 - mu) * e1 + mu * e0) / (a * a * np.sqrt(np.pi))
    I = np.prod(J)
    others = np.array([np.prod(np.delete(J, k)) for k in range(len(mu))])
    return I, others * dJmu, float(np.sum(others * dJa))


@pytest.fixture(scope="module")
def c3_grid():
    """The C3 setup: d=8, a=0.15, centres from PCG64(3); grid adapted by five
    oracle iterations, then frozen."""
    mu = W.c3_centres(3, 8)
    p = W.gauss_params(8, 0.15, mu)
    warm = oracle.run(8, 50, 3, W.GAUSS, p, [(100_000, 1)] * 5, nthreads=8)
    return warm["edges"], p


def test_gradient_matches_central_differences(c3_grid):
    """Same counters: d/dtheta of the estimator equals its central difference
    (h = 1e-4) to far better than the 1e-4 bound."""
    e, p = c3_grid
    n, it = 20_000, 5
    g = oracle.gauss_gradient(e, 3, it, n, p)
    h = 1e-4
    grad = np.concatenate([g["dmu"], [g["da"]]])
    scale = np.max(np.abs(grad))
    for c in range(9):
        idx = 1 + c if c < 8 else 0  # mu_1..mu_8, then a
        pp, pm = list(p), list(p)
        pp[idx] += h
        pm[idx] -= h
        fd = (oracle.gauss_gradient(e, 3, it, n, pp)["I"] -
              oracle.gauss_gradient(e, 3, it, n, pm)["I"]) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


def test_gradient_estimate_agrees_with_erf_derivatives(c3_grid):
    e, p = c3_grid
    g = oracle.gauss_gradient(e, 3, 9, 400_000, p)
    I, dmu, da = closed_form(p[0], p[1:])
    assert abs(g["I"] - I) < 4 * np.sqrt(g["var_I"])
    assert np.all(np.abs(g["dmu"] - dmu) < 4 * np.sqrt(g["var_dmu"]))
    assert abs(g["da"] - da) < 4 * np.sqrt(g["var_da"])


def test_gradient_value_is_the_iteration_estimate(c3_grid):
    e, p = c3_grid
    g = oracle.gauss_gradient(e, 3, 2, 5001, p)
    r = oracle.iterate(e, 3, 2, 5001, W.GAUSS, p, adapt=False)
    assert abs(g["I"] - r["I"]) <= 1e-15 * abs(r["I"])
    assert abs(g["var_I"] - r["var"]) <= 1e-12 * r["var"]


def test_closed_form_derivatives_by_differences():
    """The erf-form derivatives above against central differences of the
    closed form itself (guards the test's own formulas)."""
    a, mu = 0.15, np.array([0.3, 0.55, 0.68])
    I, dmu, da = closed_form(a, mu)
    h = 1e-6
    for k in range(3):
        up, dn = mu.copy(), mu.copy()
        up[k] += h
        dn[k] -= h
        assert abs((closed_form(a, up)[0] - closed_form(a, dn)[0]) / (2 * h) - dmu[k]) < 1e-8
    assert abs((closed_form(a + h, mu)[0] - closed_form(a - h, mu)[0]) / (2 * h) - da) < 1e-8


# ---------------------------------------------------------------- over a box
BOX = [(-1.0, 1.0), (0.0, 2.5), (0.5, 1.0), (-3.0, -1.0)]
MU_BOX = np.array([0.2, 1.1, 0.7, -2.2])


def closed_form_box(a, mu, box):
    """I = prod_k J_k over [lo_k, hi_k], J = (erf((hi-mu)/a) - erf((lo-mu)/a))/2:
    dJ/dmu = (e^{-((lo-mu)/a)^2} - e^{-((hi-mu)/a)^2}) / (a sqrt(pi)),
    dJ/da = -((hi-mu) e^{-((hi-mu)/a)^2} - (lo-mu) e^{-((lo-mu)/a)^2}) / (a^2 sqrt(pi))."""
    lo, hi = np.array(box).T
    u, v = (hi - mu) / a, (lo - mu) / a
    J = 0.5 * (erf(u) - erf(v))
    dJmu = (np.exp(-v * v) - np.exp(-u * u)) / (a * np.sqrt(np.pi))
    dJa = -((hi - mu) * np.exp(-u * u) - (lo - mu) * np.exp(-v * v)) / (a * a * np.sqrt(np.pi))
    others = np.array([np.prod(np.delete(J, k)) for k in range(len(mu))])
    return np.prod(J), others * dJmu, float(np.sum(others * dJa))


@pytest.fixture(scope="module")
def box_grid():
    p = W.gauss_params(4, 0.3, MU_BOX)
    warm = oracle.run(4, 40, 6, W.GAUSS, p, [(100_000, 1)] * 4, nthreads=8, box=BOX)
    return warm["edges"], p


def test_closed_form_over_the_unit_box_is_the_unit_cube_one():
    a, mu = 0.2, np.array([0.3, 0.55, 0.68])
    for x, y in zip(closed_form_box(a, mu, [(0.0, 1.0)] * 3), closed_form(a, mu)):
        assert np.allclose(x, y, rtol=1e-13, atol=0)


def test_boxed_gradient_is_the_chain_rule_of_the_unit_cube_one(box_grid):
    """A Gaussian (a, mu) over [lo, lo + w]^d is, sample for sample, the
    unit-cube Gaussian (a/w, (mu - lo)/w): equal I, and every derivative is the
    unit-cube one over w."""
    e, _ = box_grid
    lo, w, a = -0.4, 1.7, 0.35
    mu = np.array([0.1, 0.5, 0.9, 0.3])
    boxed = oracle.gauss_gradient(e, 4, 2, 30_000, W.gauss_params(4, a, mu),
                                  box=[(lo, lo + w)] * 4)
    unit = oracle.gauss_gradient(e, 4, 2, 30_000, W.gauss_params(4, a / w, (mu - lo) / w))
    assert abs(boxed["I"] - unit["I"]) <= 1e-12 * abs(unit["I"])
    assert np.allclose(boxed["dmu"], unit["dmu"] / w, rtol=1e-11, atol=0)
    assert abs(boxed["da"] - unit["da"] / w) <= 1e-11 * abs(unit["da"])


def test_boxed_gradient_matches_central_differences(box_grid):
    e, p = box_grid
    g = oracle.gauss_gradient(e, 6, 4, 20_000, p, box=BOX)
    grad = np.concatenate([g["dmu"], [g["da"]]])
    h, scale = 1e-4, np.max(np.abs(grad))
    for c in range(5):
        idx = 1 + c if c < 4 else 0
        pp, pm = list(p), list(p)
        pp[idx] += h
        pm[idx] -= h
        fd = (oracle.gauss_gradient(e, 6, 4, 20_000, pp, box=BOX)["I"] -
              oracle.gauss_gradient(e, 6, 4, 20_000, pm, box=BOX)["I"]) / (2 * h)
        assert abs(fd - grad[c]) <= 1e-6 * scale, (c, fd, grad[c])


def test_boxed_gradient_agrees_with_erf_derivatives_over_the_box(box_grid):
    e, p = box_grid
    g = oracle.gauss_gradient(e, 6, 9, 400_000, p, box=BOX)
    I, dmu, da = closed_form_box(p[0], MU_BOX, BOX)
    assert abs(g["I"] - I) < 4 * np.sqrt(g["var_I"])
    assert np.all(np.abs(g["dmu"] - dmu) < 4 * np.sqrt(g["var_dmu"]))
    assert abs(g["da"] - da) < 4 * np.sqrt(g["var_da"])


def test_boxed_closed_form_derivatives_by_differences():
    a, h = 0.3, 1e-6
    I, dmu, da = closed_form_box(a, MU_BOX, BOX)
    for k in range(4):
        up, dn = MU_BOX.copy(), MU_BOX.copy()
        up[k] += h
        dn[k] -= h
        fd = (closed_form_box(a, up, BOX)[0] - closed_form_box(a, dn, BOX)[0]) / (2 * h)
        assert abs(fd - dmu[k]) < 1e-8
    fd = (closed_form_box(a + h, MU_BOX, BOX)[0] - closed_form_box(a - h, MU_BOX, BOX)[0]) / (2 * h)
    assert abs(fd - da) < 1e-8
