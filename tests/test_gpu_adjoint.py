"""The adjoint kernel (vegas_gauss_adjoint) and its autograd wrapper against
the oracle's gradient, central finite differences and the analytic erf
derivatives (the d=8 setup with centres mu_i ~ U(0.3, 0.7), a = 0.15)."""
import numpy as np
import pytest

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from tests.test_oracle_gradient import closed_form  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


@pytest.fixture(scope="module")
def c3():
    """Centres from PCG64(3), a = 0.15; a grid adapted by the oracle (five
    iterations of 1e5), frozen and shared by both sides."""
    mu = W.c3_centres(3, 8)
    p = W.gauss_params(8, 0.15, mu)
    warm = oracle.run(8, 50, 3, W.GAUSS, p, [(100_000, 1)] * 5, nthreads=8)
    return warm["edges"], p


def gpu_adjoint(edges, p, mode, it, n, grad=True, seed=3):
    v = V.Vegas(8, 50, seed, mode, W.GAUSS, p, max_iters=4)
    v.set_grid(edges)
    out = v.gauss_adjoint(p, it, n, grad).cpu().numpy()
    v.close()
    return dict(I=out[0], g=out[1:10], var_I=out[10], var_g=out[11:20], bad=out[20])


def test_fp64_adjoint_matches_oracle(c3):
    e, p = c3
    o = oracle.gauss_gradient(e, 3, 5, 200_003, p)
    g = gpu_adjoint(e, p, V.VEGAS_FP64, 5, 200_003)
    og = np.concatenate([o["dmu"], [o["da"]]])
    scale = np.max(np.abs(og))
    assert abs(g["I"] - o["I"]) <= 1e-12 * abs(o["I"])
    assert np.all(np.abs(g["g"] - og) <= 1e-12 * scale)
    ov = np.concatenate([o["var_dmu"], [o["var_da"]]])
    assert np.allclose(g["var_g"], ov, rtol=1e-9)
    assert g["bad"] == 0


@pytest.mark.parametrize("dim", [1, 3, 13, 20])
def test_fp64_adjoint_matches_oracle_across_dims(dim):
    """Every dimension the kernels are built for, on a random monotone grid:
    I and dI/d(mu, a) equal the oracle's to 1e-12 (same counters), the
    variances to 1e-9."""
    rng = np.random.Generator(np.random.PCG64(dim))
    p = W.gauss_params(dim, 0.25, rng.uniform(0.3, 0.7, dim))
    e = W.random_monotone_grid(dim, 30, seed=dim, spread=0.5)
    o = oracle.gauss_gradient(e, 7, 2, 100_001, p)
    v = V.Vegas(dim, 30, 7, V.VEGAS_FP64, W.GAUSS, p, max_iters=4)
    v.set_grid(e)
    out = v.gauss_adjoint(p, 2, 100_001, True).cpu().numpy()
    v.close()
    nc = dim + 1
    og = np.concatenate([o["dmu"], [o["da"]]])
    assert abs(out[0] - o["I"]) <= 1e-12 * abs(o["I"])
    assert np.all(np.abs(out[1:1 + nc] - og) <= 1e-12 * np.max(np.abs(og)))
    ov = np.concatenate([o["var_dmu"], [o["var_da"]]])
    assert np.allclose(out[2 + nc:2 + 2 * nc], ov, rtol=1e-9)
    assert out[2 * nc + 2] == 0


def test_fp32_adjoint_within_its_error_budget(c3):
    """Same counters in float: every component within 1% of its own Monte
    Carlo error of the FP64 oracle (the float rounding is far below it)."""
    e, p = c3
    o = oracle.gauss_gradient(e, 3, 5, 200_003, p)
    g = gpu_adjoint(e, p, V.VEGAS_FP32_EVAL, 5, 200_003)
    og = np.concatenate([o["dmu"], [o["da"]]])
    sg = np.sqrt(np.concatenate([o["var_dmu"], [o["var_da"]]]))
    assert abs(g["I"] - o["I"]) <= 0.01 * np.sqrt(o["var_I"])
    assert np.all(np.abs(g["g"] - og) <= 0.01 * sg)


@pytest.mark.parametrize("dim", [3, 12, 16, 17])
def test_fp32_adjoint_at_50_bins_across_dims(dim):
    """Float adjoints at 50 bins (the kernels compiled for that bin count up to
    d = 16; d = 17 takes the general one) on a random monotone grid: I and
    every gradient component within 1% of its own Monte Carlo error of the
    FP64 oracle's on the same counters, in both the gradient and the
    value-only call."""
    rng = np.random.Generator(np.random.PCG64(100 + dim))
    p = W.gauss_params(dim, 0.25, rng.uniform(0.3, 0.7, dim))
    e = W.random_monotone_grid(dim, 50, seed=dim, spread=0.5)
    n = 200_003
    o = oracle.gauss_gradient(e, 7, 2, n, p)
    v = V.Vegas(dim, 50, 7, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=4)
    v.set_grid(e)
    out = v.gauss_adjoint(p, 2, n, True).cpu().numpy()
    val = v.gauss_adjoint(p, 2, n, False).cpu().numpy()
    v.close()
    nc = dim + 1
    og = np.concatenate([o["dmu"], [o["da"]]])
    sg = np.sqrt(np.concatenate([o["var_dmu"], [o["var_da"]]]))
    assert abs(out[0] - o["I"]) <= 0.01 * np.sqrt(o["var_I"])
    assert np.all(np.abs(out[1:1 + nc] - og) <= 0.01 * sg)
    assert abs(val[0] - o["I"]) <= 0.01 * np.sqrt(o["var_I"])
    assert out[2 * nc + 2] == 0 and val[2 * nc + 2] == 0


def test_value_only_call(c3):
    e, p = c3
    g = gpu_adjoint(e, p, V.VEGAS_FP64, 1, 10_000, grad=False)
    r = oracle.iterate(e, 3, 1, 10_000, W.GAUSS, p, adapt=False)
    assert abs(g["I"] - r["I"]) <= 1e-12 * abs(r["I"])
    assert np.all(g["g"] == 0.0) and abs(g["var_I"] - r["var"]) <= 1e-10 * r["var"]


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_full_size_gradient_vs_analytic_and_differences(c3, mode):
    """1e8 samples recomputed from their counters: the gradient agrees with
    the erf derivatives within 4 sigma, and (FP64) with central differences
    of the same estimator (h = 1e-4) to 1e-4 relative."""
    e, p = c3
    n = 100_000_000
    v = V.Vegas(8, 50, 3, mode, W.GAUSS, p, max_iters=4)
    v.set_grid(e)
    out = v.gauss_adjoint(p, 7, n, True).cpu().numpy()
    I, dmu, da = closed_form(p[0], p[1:])
    exact = np.concatenate([dmu, [da]])
    assert abs(out[0] - I) < 4 * np.sqrt(out[10])
    assert np.all(np.abs(out[1:10] - exact) < 4 * np.sqrt(out[11:20]))
    if mode == V.VEGAS_FP64:
        h, scale = 1e-4, np.max(np.abs(out[1:10]))
        for c in range(9):
            idx = 1 + c if c < 8 else 0
            pp, pm = list(p), list(p)
            pp[idx] += h
            pm[idx] -= h
            fp = v.gauss_adjoint(pp, 7, n, False).cpu().numpy()[0]
            fm = v.gauss_adjoint(pm, 7, n, False).cpu().numpy()[0]
            assert abs((fp - fm) / (2 * h) - out[1 + c]) <= 1e-4 * scale, c
    v.close()


def test_autograd_function(c3):
    from paper_2002_12921_b300.autodiff import gauss_integral

    e, p = c3
    v = V.Vegas(8, 50, 3, V.VEGAS_FP64, W.GAUSS, p, max_iters=4)
    v.set_grid(e)
    mu = torch.tensor(p[1:], dtype=torch.float64, device="cuda", requires_grad=True)
    a = torch.tensor(p[0], dtype=torch.float64, requires_grad=True)
    I = gauss_integral(mu, a, v, 5, 200_003)
    gmu, ga = torch.autograd.grad(3.0 * I, (mu, a))
    o = oracle.gauss_gradient(e, 3, 5, 200_003, p)
    scale = np.max(np.abs(o["dmu"]))
    assert abs(I.item() - o["I"]) <= 1e-12
    assert np.all(np.abs(gmu.cpu().numpy() - 3.0 * o["dmu"]) <= 3e-12 * scale)
    assert abs(ga.item() - 3.0 * o["da"]) <= 3e-12 * abs(o["da"])
    assert gmu.device == mu.device and ga.device == a.device
    v.close()
