"""Integration over a box [lo_k, hi_k] (vegas_set_box): the grid stays in unit
coordinates u, samples are evaluated at x = lo + (hi - lo) u and weighted by
the extra Jacobian prod (hi - lo).

FP64 runs match the oracle's boxed runs within the FP64 parity bounds, FP32
first iterations the oracle's within the float bound; the unit box reproduces
the unit cube up to summation order; the change of variables of a Gaussian gives the
unit-cube sums; caller-compiled integrands reach their closed forms over a box;
misuse is refused, checkpoints carry the box, and the adjoint differentiates the
boxed integral."""
import os
from math import erf

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


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


def fp64_tol(edges):
    """As in the unit-cube parity tests: an edge that both sides refined to one
    ulp moves a width Delta by eps/Delta relative, over d dimensions."""
    dmin = np.min(np.diff(edges, axis=1))
    return max(RTOL64, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def boxed_run(dim, nbins, seed, fid, params, box, schedule, mode, alpha=1.5):
    v = V.Vegas(dim, nbins, seed, mode, fid, params, max_iters=len(schedule) + 2)
    v.set_box(box)
    grids = []
    for n, adapt in schedule:
        grids.append(v.grid())
        v.iterate(n, adapt)
        if adapt:
            v.refine(alpha)
    rows, edges = v.iterations(), v.grid()
    v.close()
    return rows, grids, edges


BOXES = {
    "gauss4": (W.GAUSS, 4, 40, [(-1.0, 1.0), (0.0, 3.0), (-2.0, 0.5), (10.0, 10.25)],
               lambda: W.gauss_params(4, 0.3, [0.2, 1.0, -0.5, 10.1])),
    "mix6": (W.GAUSS_MIX2, 6, 50, [(-0.5, 1.5)] * 6, lambda: W.mix2_params(6, 0.2)),
    "ppeak5": (W.GENZ_PPEAK, 5, 30, [(0.25, 0.75), (0.0, 2.0), (-1.0, 1.0), (0.5, 0.6),
                                     (0.0, 1.0)],
               lambda: W.genz_params(5, seed=5, kind=W.GENZ_PPEAK)),
    "flat3": (W.FLAT, 3, 16, [(-1.0, 2.0), (0.25, 0.5), (3.0, 10.0)], lambda: []),
}


@pytest.mark.parametrize("case", sorted(BOXES))
def test_fp64_boxed_run_matches_oracle(case):
    fid, dim, nbins, box, params = BOXES[case]
    p = params()
    sched = [(30_011, 1), (20_000, 1), (12_345, 0)]
    rows, grids, edges = boxed_run(dim, nbins, 21, fid, p, box, sched, V.VEGAS_FP64)
    o = oracle.run(dim, nbins, 21, fid, p, sched, nthreads=8, box=box)
    for t, (n, adapt) in enumerate(sched):
        ref = o["log"][t]
        tol = RTOL64 if t == 0 else fp64_tol(o["grids"][t])
        assert rows[t][2] == n
        assert abs(rows[t][4] - ref["I"]) <= tol * abs(ref["I"]), (t, rows[t][4], ref["I"])
        assert abs(rows[t][5] - ref["var"]) <= 100 * tol * abs(ref["var"]) + 1e-300, t
        etol = RTOL64 if t == 0 else max(RTOL64, 2 * fp64_tol(o["grids"][t - 1]))
        assert np.allclose(grids[t], o["grids"][t], rtol=etol, atol=1e-15), t
    assert np.allclose(edges, o["edges"], rtol=max(RTOL64, 2 * fp64_tol(o["grids"][1])),
                       atol=1e-15)


@pytest.mark.parametrize("case,tol", [("gauss4", 1e-5), ("mix6", 1e-5), ("ppeak5", 1e-5)])
def test_fp32_boxed_first_iteration_within_float_bound(case, tol):
    fid, dim, nbins, box, params = BOXES[case]
    p = params()
    warm = oracle.run(dim, nbins, 99, fid, p, [(100_000, 1)] * 3, nthreads=8, box=box)
    e = warm["edges"]
    o = oracle.iterate(e, 7, 0, 400_000, fid, p, adapt=True, nthreads=8, box=box)
    v = V.Vegas(dim, nbins, 7, V.VEGAS_FP32_EVAL, fid, p, max_iters=4)
    v.set_grid(e)
    v.set_box(box)
    v.iterate(400_000, 1)
    row, h = v.iterations()[0], v.histogram()
    v.close()
    assert abs(row[4] - o["I"]) <= tol * abs(o["I"])
    assert abs(row[5] - o["var"]) <= 10 * tol * (o["var"] + o["I"] ** 2 / 400_000)
    assert np.allclose(h.sum(axis=1), o["hist"].sum(axis=1), rtol=10 * tol)


# two runs of the same state agree up to the order of the device's atomic
# sums: ~1e-13 in FP64; in FP32 a grid that moved by an ulp can round a staged
# float the other way, which moves I by a float rounding
SAME_RUN_TOL = {V.VEGAS_FP64: 1e-13, V.VEGAS_FP32_EVAL: 1e-5}


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_unit_box_reproduces_the_unit_cube(mode):
    """lo = 0, hi = 1 leaves every staged constant unchanged (x 1 + 0): the
    first iteration is the unit cube's up to summation order, and so are the
    later ones."""
    p = W.gauss_params(6, 0.15, np.linspace(0.3, 0.7, 6))
    sched = [(100_000, 1)] * 3 + [(80_000, 0)]
    out = []
    for box in (None, [(0.0, 1.0)] * 6):
        v = V.Vegas(6, 30, 4, mode, W.GAUSS, p, max_iters=8)
        if box is not None:
            v.set_box(box)
        v.run(sched)
        out.append((v.iterations(), v.grid()))
        v.close()
    tol = SAME_RUN_TOL[mode]
    # rows: S1, S2, n, nonfinite, I, var
    assert np.array_equal(out[0][0][:, 2:4], out[1][0][:, 2:4])
    assert np.allclose(out[0][0][:, 4], out[1][0][:, 4], rtol=tol, atol=0)
    assert np.allclose(out[0][0][0], out[1][0][0], rtol=1e-13, atol=0)
    assert np.allclose(out[0][1], out[1][1], rtol=0, atol=10 * tol)


def test_gaussian_over_a_box_is_the_unit_cube_change_of_variables():
    """A Gaussian (a, mu) over [lo, lo + w]^d is the unit-cube Gaussian with
    a / w and (mu - lo) / w, sample for sample (FP64)."""
    lo, w, a = -0.7, 2.5, 0.4
    mu = np.array([0.1, 0.5, 1.2])
    sched = [(60_000, 1)] * 2 + [(40_000, 0)]
    rows_b, _, edges_b = boxed_run(3, 25, 3, W.GAUSS, W.gauss_params(3, a, mu),
                                   [(lo, lo + w)] * 3, sched, V.VEGAS_FP64)
    v = V.Vegas(3, 25, 3, V.VEGAS_FP64, W.GAUSS, W.gauss_params(3, a / w, (mu - lo) / w),
                max_iters=8)
    v.run(sched)
    rows_u, edges_u = v.iterations(), v.grid()
    v.close()
    assert np.allclose(rows_b[:, 4], rows_u[:, 4], rtol=1e-11, atol=0)
    assert np.allclose(edges_b, edges_u, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_boxed_gaussian_reaches_the_erf_closed_form(mode):
    box = [(-1.0, 1.0), (0.0, 3.0), (-2.0, 0.5), (0.0, 1.0)]
    mu, a = np.array([0.2, 1.0, -0.5, 0.5]), 0.3
    exact = float(np.prod([0.5 * (erf((hi - m) / a) - erf((lo - m) / a))
                           for (lo, hi), m in zip(box, mu)]))
    v = V.Vegas(4, 50, 11, mode, W.GAUSS, W.gauss_params(4, a, mu), max_iters=12)
    v.set_box(box)
    v.run([(500_000, 1)] * 6 + [(2_000_000, 0)] * 3)
    mean, sigma, chi2, k, bad = v.result(6)
    v.close()
    assert k == 9 and not bad
    assert sigma < 1e-3 * exact
    assert abs(mean - exact) < 5 * sigma, (mean, sigma, exact)


@pytest.fixture(scope="module")
def user_so():
    return build.build_user_integrand(os.path.join(ROOT, "tests", "user_integrands.cu"),
                                      os.path.join(ROOT, "tests", "_build",
                                                   "libuser_integrands.so"))


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_user_integrand_over_a_box_reaches_its_closed_form(user_so, mode):
    """(sum_k x_k)^2 over prod [lo_k, hi_k]: with m_k, v_k the mean and variance
    of the uniform x_k, the integral is vol ((sum m_k)^2 + sum v_k)."""
    box = [(-1.0, 1.0), (0.5, 2.0), (0.0, 0.25), (-3.0, -1.0), (1.0, 4.0)]
    lo, hi = np.array(box).T
    m, var = (lo + hi) / 2, (hi - lo) ** 2 / 12
    exact = float(np.prod(hi - lo) * (m.sum() ** 2 + var.sum()))
    mod, desc = V.load_user_integrand(user_so, "user_sum_square_d5")
    v = V.Vegas(5, 50, 99, mode, V.VEGAS_USER, None, max_iters=12)
    v.set_user_integrand(desc, None, mod)
    v.set_box(box)
    v.run([(200_000, 1)] * 5 + [(1_000_000, 0)] * 3)
    mean, sigma, chi2, k, bad = v.result(5)
    v.close()
    assert k == 8 and not bad
    assert sigma < 1e-3 * abs(exact)
    assert abs(mean - exact) < 5 * sigma, (mean, sigma, exact)


def test_misuse_is_refused():
    p = W.gauss_params(3, 0.2)
    v = V.Vegas(3, 20, 1, V.VEGAS_FP64, W.GAUSS, p, max_iters=4)
    for bad in ([(0.0, 1.0), (1.0, 1.0), (0.0, 1.0)],          # empty interval
                [(0.0, 1.0), (2.0, 1.0), (0.0, 1.0)],          # hi < lo
                [(0.0, np.inf)] * 3, [(np.nan, 1.0)] * 3):
        with pytest.raises(V.VegasError) as e:
            v.set_box(bad)
        assert e.value.status == V.VEGAS_EINVAL
    v.set_box([(0.0, 2.0)] * 3)
    v.iterate(1000, 1)
    with pytest.raises(V.VegasError) as e:                      # only before iterating
        v.set_box([(0.0, 3.0)] * 3)
    assert e.value.status == V.VEGAS_ESTATE
    v.close()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_checkpoint_carries_the_box(mode):
    p = W.gauss_params(4, 0.25, [0.0, 1.0, 2.0, -1.0])
    box = [(-1.0, 1.0), (0.0, 2.0), (1.0, 3.0), (-2.0, 0.0)]
    a = V.Vegas(4, 30, 8, mode, W.GAUSS, p, max_iters=8)
    a.set_box(box)
    a.run([(100_000, 1)] * 2)
    blob = a.export_state()
    b = V.Vegas.from_state(blob)
    for v in (a, b):
        v.run([(100_000, 1), (150_000, 0)])
    ra, rb = a.iterations(), b.iterations()
    assert np.array_equal(ra[:2], rb[:2])                       # the log came along
    tol = SAME_RUN_TOL[mode]                                    # and the box: same I
    assert np.allclose(rb[:, 4], ra[:, 4], rtol=tol, atol=0)
    assert np.allclose(b.grid(), a.grid(), rtol=0, atol=10 * tol)
    a.close()
    b.close()


def test_virtual_ranks_over_a_box_equal_the_oracle():
    """A boxed integral sharded over 3 virtual ranks (counter ranges, summed
    partials, every rank refining) equals the oracle's boxed run (FP64)."""
    from paper_2002_12921_b300.shard import GpuShardEngine, VirtualRanks

    fid, dim, nbins, box, params = BOXES["gauss4"]
    p = params()
    sched = [(90_001, 1), (60_000, 1), (50_000, 0)]
    states = []
    for _ in range(3):
        s = V.Vegas(dim, nbins, 13, V.VEGAS_FP64, fid, p, max_iters=8)
        s.set_box(box)
        states.append(s)
    VirtualRanks([GpuShardEngine(s) for s in states]).run(sched)
    o = oracle.run(dim, nbins, 13, fid, p, sched, nthreads=8, box=box)
    for s in states:
        rows = s.iterations()
        for t, ref in enumerate(o["log"]):
            tol = RTOL64 if t == 0 else fp64_tol(o["grids"][t])
            assert abs(rows[t][4] - ref["I"]) <= tol * abs(ref["I"]), t
        assert np.allclose(s.grid(), o["edges"], rtol=max(RTOL64, 2 * fp64_tol(o["grids"][1])),
                           atol=1e-15)
        s.close()


@pytest.mark.parametrize("mode,tol", [(V.VEGAS_FP64, None), (V.VEGAS_FP32_EVAL, 0.01)])
def test_adjoint_over_a_box_matches_the_oracle(mode, tol):
    """dI/d(mu, a) of a boxed Gaussian on a frozen grid: FP64 equal to the
    oracle's boxed gradient to 1e-12 (same counters), FP32 within 1% of each
    component's Monte Carlo error."""
    box = [(-1.0, 1.0), (0.0, 2.5), (0.5, 1.0), (-3.0, -1.0)]
    p = W.gauss_params(4, 0.3, [0.2, 1.1, 0.7, -2.2])
    e = oracle.run(4, 40, 6, W.GAUSS, p, [(100_000, 1)] * 4, nthreads=8, box=box)["edges"]
    o = oracle.gauss_gradient(e, 6, 4, 200_003, p, box=box)
    v = V.Vegas(4, 40, 6, mode, W.GAUSS, p, max_iters=4)
    v.set_grid(e)
    v.set_box(box)
    out = v.gauss_adjoint(p, 4, 200_003).cpu().numpy()
    v.close()
    og = np.concatenate([[o["I"]], o["dmu"], [o["da"]]])
    if tol is None:
        assert np.all(np.abs(out[:6] - og) <= 1e-12 * np.max(np.abs(og)))
        ov = np.concatenate([[o["var_I"]], o["var_dmu"], [o["var_da"]]])
        assert np.allclose(out[6:12], ov, rtol=1e-9)
    else:
        sg = np.sqrt(np.concatenate([[o["var_I"]], o["var_dmu"], [o["var_da"]]]))
        assert np.all(np.abs(out[:6] - og) <= tol * sg)
    assert out[12] == 0


@pytest.mark.parametrize("dim,nbins,box", [
    (20, 50, [(-0.5 - 0.05 * k, 1.0 + 0.1 * k) for k in range(20)]),   # the largest dimension
    (3, 1, [(2.0, 5.0), (-1.0, 0.0), (0.0, 0.125)]),                  # one bin: plain MC
    (2, 40, [(1e3, 1e3 + 1e-3), (-7.5, -7.25)]),                       # narrow, far from 0
])
def test_fp64_boxed_edge_cases_match_oracle(dim, nbins, box):
    lo, hi = np.array(box).T
    p = W.gauss_params(dim, 0.5, (lo + hi) / 2 + 0.1 * (hi - lo))
    if dim == 2:
        p = W.gauss_params(dim, 1e-3, (lo + hi) / 2)
    sched = [(20_011, 1), (20_011, 1), (10_000, 0)]
    rows, grids, edges = boxed_run(dim, nbins, 33, W.GAUSS, p, box, sched, V.VEGAS_FP64)
    o = oracle.run(dim, nbins, 33, W.GAUSS, p, sched, nthreads=8, box=box)
    for t, ref in enumerate(o["log"]):
        tol = RTOL64 if t == 0 else fp64_tol(o["grids"][t])
        if dim == 2:
            # x = lo + w u near 1e3 carries eps |x| of rounding on either side,
            # which z = (x - mu)/a magnifies by 1/a: f = e^{-z^2} moves by
            # 2 |z| dz relative, and samples with |z| > 6 carry less than
            # e^-36 of I, so the bound is sum_k 4 * 6 eps |x_k|max / a, with
            # no averaging over samples assumed
            xmax = np.maximum(np.abs(lo), np.abs(hi))
            tol = max(tol, np.sum(24 * np.finfo(float).eps * xmax / p[0]))
        assert abs(rows[t][4] - ref["I"]) <= tol * abs(ref["I"]), (t, rows[t][4], ref["I"])
    assert np.all(np.diff(edges, axis=1) > 0)
