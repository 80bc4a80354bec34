"""Integrands compiled by the caller (include/vegas_user_integrand.cuh, the
VEGAS_USER integrand id) through the C ABI.

tests/user_integrands.cu writes the Eq. 1 Gaussian in the plain coordinate
with its parameters in caller device memory: in FP64 it must reproduce the
oracle's Gaussian run (same counters, same samples) within the FP64 parity
bounds, in FP32 the oracle's first iteration within the float bound.  Two
integrands the library does not build in, a non-separable (sum x_k)^2 and a
product of sines, must reach their closed forms."""
import ctypes
import os

import numpy as np
import pytest

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import build
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
RTOL64 = 1e-12


@pytest.fixture(scope="module")
def so():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()
    return build.build_user_integrand(os.path.join(ROOT, "tests", "user_integrands.cu"),
                                      os.path.join(ROOT, "tests", "_build",
                                                   "libuser_integrands.so"))


def user_state(so, name, dim, nbins, seed, mode, data=None, max_iters=16):
    mod, desc = V.load_user_integrand(so, name)
    v = V.Vegas(dim, nbins, seed, mode, V.VEGAS_USER, None, max_iters=max_iters)
    v.set_user_integrand(desc, data, mod)
    return v


def fp64_tol(edges):
    dmin = np.min(np.diff(edges, axis=1))
    return max(RTOL64, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def run(v, schedule, alpha=1.5):
    grids = []
    for n, adapt in schedule:
        grids.append(v.grid())
        v.iterate(n, adapt)
        if adapt:
            v.refine(alpha)
    return grids, v.iterations()


@pytest.mark.parametrize("name,dim", [("user_gauss_d4", 4), ("user_gauss_d8", 8)])
def test_fp64_user_gauss_matches_oracle_gauss(so, name, dim):
    p = W.gauss_params(dim, 0.2, np.linspace(0.35, 0.65, dim))
    data = torch.tensor(p, dtype=torch.float64, device="cuda")
    sched = [(20011, 1)] * 3 + [(20011, 0)]
    v = user_state(so, name, dim, 40, 123, V.VEGAS_FP64, data)
    grids, rows = run(v, sched)
    o = oracle.run(dim, 40, 123, W.GAUSS, p, sched, nthreads=4)
    for t in range(len(sched)):
        tol = RTOL64 if t == 0 else fp64_tol(o["grids"][t])
        assert rows[t][2] == sched[t][0]
        assert abs(rows[t][4] - o["log"][t]["I"]) <= tol * abs(o["log"][t]["I"]), t
        assert abs(rows[t][5] - o["log"][t]["var"]) <= 100 * tol * o["log"][t]["var"], t
        assert np.allclose(grids[t], o["grids"][t], rtol=RTOL64, atol=1e-15), t
    assert np.allclose(v.grid(), o["edges"], rtol=RTOL64, atol=1e-15)
    v.close()


def test_fp32_user_gauss_first_iteration_within_float_bound(so):
    dim = 8
    p = W.gauss_params(dim, 0.25, np.full(dim, 0.5))
    data = torch.tensor(p, dtype=torch.float64, device="cuda")
    v = user_state(so, "user_gauss_d8", dim, 50, 7, V.VEGAS_FP32_EVAL, data)
    v.iterate(100_003, 0)
    row = v.iterations()[0]
    o = oracle.run(dim, 50, 7, W.GAUSS, p, [(100_003, 0)], nthreads=4)
    assert abs(row[4] - o["log"][0]["I"]) <= 1e-5 * o["log"][0]["I"]
    assert abs(row[5] - o["log"][0]["var"]) <= 1e-4 * o["log"][0]["var"]
    v.close()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
@pytest.mark.parametrize("name,dim,exact", [("user_sum_square_d5", 5, 5 / 12 + 25 / 4),
                                            ("user_sine_d3", 3, 1.0)])
def test_closed_forms(so, mode, name, dim, exact):
    v = user_state(so, name, dim, 50, 99, mode)
    v.run([(200_000, 1)] * 5 + [(1_000_000, 0)] * 3)
    mean, sigma, chi2, k, bad = v.result(5)  # combined over iterations 5..7
    assert k == 8 and not bad
    assert sigma < 1e-3 * exact
    assert abs(mean - exact) < 5 * sigma, (mean, sigma, exact)
    v.close()


def test_user_gauss_equals_builtin_gauss(so):
    """The same seed drives the same grid mechanics: the adapting user
    Gaussian and the built-in one refine to the same grid (FP64)."""
    dim = 4
    p = W.gauss_params(dim, 0.15, np.array([0.3, 0.4, 0.6, 0.7]))
    data = torch.tensor(p, dtype=torch.float64, device="cuda")
    u = user_state(so, "user_gauss_d4", dim, 30, 5, V.VEGAS_FP64, data)
    b = V.Vegas(dim, 30, 5, V.VEGAS_FP64, V.VEGAS_GAUSS, p, max_iters=16)
    sched = [(50_000, 1)] * 2
    u.run(sched)
    b.run(sched)
    ru, rb = u.iterations(), b.iterations()
    assert np.allclose(ru[:, 4], rb[:, 4], rtol=1e-12, atol=0)
    assert np.allclose(u.grid(), b.grid(), rtol=1e-12, atol=1e-15)
    u.close()
    b.close()


def test_errors_and_checkpoint(so):
    dim = 4
    p = W.gauss_params(dim, 0.2, np.full(dim, 0.5))
    data = torch.tensor(p, dtype=torch.float64, device="cuda")
    mod, d4 = V.load_user_integrand(so, "user_gauss_d4")
    _, d8 = V.load_user_integrand(so, "user_gauss_d8")
    # a built-in state takes no user kernels; a dimension mismatch is refused
    b = V.Vegas(dim, 20, 1, V.VEGAS_FP64, V.VEGAS_GAUSS, p, max_iters=4)
    with pytest.raises(V.VegasError) as e:
        b.set_user_integrand(d4, data, mod)
    assert e.value.status == V.VEGAS_EINVAL
    b.close()
    u = V.Vegas(dim, 20, 1, V.VEGAS_FP64, V.VEGAS_USER, None, max_iters=8)
    with pytest.raises(V.VegasError) as e:
        u.set_user_integrand(d8, data, mod)
    assert e.value.status == V.VEGAS_EINVAL
    # iterating before the kernels are attached is a state error
    with pytest.raises(V.VegasError) as e:
        u.iterate(1000, 1)
    assert e.value.status == V.VEGAS_ESTATE
    # a user state checkpoints like any other; the restored one needs the
    # kernels again and then continues exactly
    u.set_user_integrand(d4, data, mod)
    u.run([(30_000, 1)] * 2)
    blob = u.export_state()
    u.run([(30_000, 1)] * 2)
    r = V.Vegas.from_state(blob)
    with pytest.raises(V.VegasError) as e:
        r.iterate(30_000, 1)
    assert e.value.status == V.VEGAS_ESTATE
    r.set_user_integrand(d4, data, mod)
    r.run([(30_000, 1)] * 2)
    # the same samples; the histogram's atomic FP64 sums differ in order only
    ru, rr = u.iterations(), r.iterations()
    assert np.array_equal(rr[:2], ru[:2]) and np.array_equal(rr[:, 2], ru[:, 2])
    assert np.allclose(rr[:, 4], ru[:, 4], rtol=1e-12, atol=0)
    assert np.allclose(r.grid(), u.grid(), rtol=0, atol=1e-14)
    u.close()
    r.close()
    assert ctypes.sizeof(V.vegas_user_integrand) >= 24


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_nonfinite_user_values_are_counted_and_left_out(so, mode):
    """NaN where x_1 < 1/4, 1 elsewhere, on the uniform 4-bin grid: the bad
    samples are those whose first Philox word is below 2^30 (bin 0 of
    dimension 1), counted here from the oracle's words.  The iteration must
    report exactly that many non-finite values, the estimate (n - bad)/n, and
    a histogram holding each finite sample's (f J)^2 = 1 in its bins."""
    n, seed = 100_003, 21
    v = user_state(so, "user_hole_d2", 2, 4, seed, mode)
    v.iterate(n, 1)
    row, hist = v.iterations()[0], v.histogram()
    v.close()
    i = np.arange(n, dtype=np.uint64)
    ctrs = np.stack([(i & 0xFFFFFFFF).astype(np.uint32), (i >> 32).astype(np.uint32),
                     np.zeros(n, np.uint32), np.zeros(n, np.uint32)], axis=1)
    w = oracle.philox(ctrs, np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32))
    bins = (w[:, :2].astype(np.uint64) * 4) >> 32
    bad = int(np.sum(bins[:, 0] == 0))
    assert row[3] == bad
    assert row[0] == n - bad and row[4] == (n - bad) / n
    ok = bins[:, 0] != 0
    for k in range(2):
        assert np.array_equal(hist[k], np.bincount(bins[ok, k].astype(np.int64), minlength=4))
