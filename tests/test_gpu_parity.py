"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 mode: the same counters give the same samples, so per-iteration I, var,
the histogram and the refined grid agree with the oracle to 1e-12 relative (the
only differences are rounding order and 1-ulp differences of exp).
FP32-eval mode: compared on the same grid and counters within the float
error budget (|dI| <= 1e-5 |I|, |dvar| <= 1e-4 var for d <= 8; 3x that at
d = 16), and statistically (3 sigma) over whole runs.
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

from tests.fp32_budget import assert_hist_close, fp32_hist_tol, prescale_h

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


def gpu_run(wl_dim, nbins, seed, fid, params, schedule, mode, alpha=1.5, edges=None, cfg=None,
            max_iters=64, first_iter=0):
    v = V.Vegas(wl_dim, nbins, seed, mode, fid, params, max_iters=max_iters)
    if cfg:
        v.config(**cfg)
    if edges is not None:
        v.set_grid(edges)
    grids, hists = [], []
    for n, adapt in schedule:
        grids.append(v.grid())
        v.iterate(n, adapt)
        if adapt:
            hists.append(v.histogram())
            v.refine(alpha)
    rows = v.iterations()
    final = v.grid()
    res = v.result(first_iter)
    v.close()
    return dict(rows=rows, grids=grids, hists=hists, edges=final, result=res)


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300))


def fp64_tol(edges):
    """Relative tolerance of I in FP64 mode on a grid that both sides refined.
    The two refinements agree to about one ulp of the edges, and a width
    Delta = e_{j+1} - e_j then carries a relative error of eps/Delta, which the
    Jacobian prod_k N Delta_k accumulates over the d dimensions: bound
    8 d eps / min Delta, and never below the 1e-12 target."""
    dmin = np.min(np.diff(edges, axis=1))
    return max(RTOL64, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def assert_fp64_parity(g, o, schedule):
    for t, (n, adapt) in enumerate(schedule):
        row, ref = g["rows"][t], o["log"][t]
        tol = fp64_tol(o["grids"][t]) if t > 0 else RTOL64
        assert row[2] == n
        assert rel(row[4], ref["I"]) < tol, (t, row[4], ref["I"], tol)
        assert rel(row[5], ref["var"]) < 100 * tol, (t, row[5], ref["var"], tol)
        assert row[3] == ref["nonfinite"]
        # grid t was refined from iteration t-1's histogram of (f J)^2, whose
        # relative error is twice that iteration's bound on f J
        etol = RTOL64 if t == 0 else max(RTOL64, 2 * fp64_tol(o["grids"][t - 1]))
        assert np.allclose(g["grids"][t], o["grids"][t], rtol=etol, atol=1e-15), t
    k, etol = 0, RTOL64
    for t, (n, adapt) in enumerate(schedule):
        if adapt:
            # (f J)^2 carries twice the relative error bound of f J on grid t
            htol = max(1e-11, 2 * fp64_tol(o["grids"][t]))
            assert np.allclose(g["hists"][k], o["log"][t]["hist"], rtol=htol, atol=0), t
            etol = max(RTOL64, 2 * fp64_tol(o["grids"][t]))
            k += 1
    # the final grid was refined from the last adapting iteration's histogram
    assert np.allclose(g["edges"], o["edges"], rtol=etol, atol=1e-15)


# ---------------------------------------------------------------- RNG
def test_philox_words_bit_exact():
    """GPU Philox words == oracle words on counters that cross the 32-bit carry
    of the sample index, for several dims, iterations and integral ids."""
    for seed, ident, it, i0, n, dim in [(1, 0, 0, 0, 4096, 8), (0xDEADBEEF12345678, 3, 7,
                                        2**32 - 1000, 2000, 5), (2**64 - 1, 255, 2**32 - 1, 2**40,
                                        700, 16), (42, 1, 1, 12345, 1001, 1),
                                       (7, 9, 3, 2**32 - 500, 1000, 20)]:
        out = torch.empty((n, dim), dtype=torch.int32, device="cuda")
        V.vegas_sample_words(seed, ident, it, i0, n, dim, out.data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32)
        sel = np.unique(np.concatenate([np.arange(0, n, 7), [n - 1]]))
        ref = np.array([oracle.sample_words(seed, ident, it, i0 + int(r), dim) for r in sel])
        assert np.array_equal(got[sel], ref)


def test_philox_words_bulk_1e6():
    n, dim = 1 << 18, 4
    out = torch.empty((n, dim), dtype=torch.int32, device="cuda")
    V.vegas_sample_words(9, 0, 3, 2**32 - n // 2, n, dim, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy().view(np.uint32)
    i = 2**32 - n // 2 + np.arange(n, dtype=np.uint64)
    ctrs = np.stack([(i & 0xFFFFFFFF).astype(np.uint32), (i >> 32).astype(np.uint32),
                     np.zeros(n, np.uint32), np.full(n, 3, np.uint32)], axis=1)
    ref = oracle.philox(ctrs, np.array([9, 0], dtype=np.uint32))
    assert np.array_equal(got, ref)


def test_philox_words_equal_curand_philox4_32_10():
    """The library's words equal cuRAND's Philox4_32_10 (device API, a second
    implementation) at the same key and counter: sample i, call q of iteration
    t is cuRAND subsequence t << 32 | (q | integral_id << 8) at offset 4 i.
    Counters cross the 32-bit carry of the sample index; dims 16 use all four
    calls."""
    import ctypes
    import os

    from paper_2002_12921_b300 import build

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = build.build_module(os.path.join(root, "tests", "curand_philox.cu"),
                            os.path.join(root, "tests", "_build", "libcurand_philox.so"))
    cr = ctypes.CDLL(so)
    cr.curand_philox_words.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p,
                                       ctypes.c_void_p]
    stream = torch.cuda.current_stream().cuda_stream
    for seed, ident, it, i0, n in [(2, 0, 0, 0, 50_000), (0xDEADBEEF12345678, 3, 7, 2**32 - 20_000,
                                   40_000), (2**64 - 1, 255, 2**32 - 1, 2**40, 10_000)]:
        dim = 16
        ours = torch.empty((n, dim), dtype=torch.int32, device="cuda")
        V.vegas_sample_words(seed, ident, it, i0, n, dim, ours.data_ptr(), stream)
        for q in range(4):
            ref = torch.empty((n, 4), dtype=torch.int32, device="cuda")
            assert cr.curand_philox_words(seed, q | ident << 8, it, i0, n, ref.data_ptr(),
                                          stream) == 0
            torch.cuda.synchronize()
            assert torch.equal(ours[:, 4 * q:4 * q + 4], ref), (seed, q)


def test_fp64_exp_within_two_ulp_of_exp_everywhere():
    """The FP64 integrands' table-driven exponential against the CUDA library's
    exp and numpy's on the whole argument range, including the subnormal
    results, the overflow and underflow thresholds and special values."""
    import ctypes
    import os

    from paper_2002_12921_b300 import build

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    so = build.build_module(os.path.join(root, "tests", "fp64_exp_check.cu"),
                            os.path.join(root, "tests", "_build", "libfp64_exp_check.so"))
    m = ctypes.CDLL(so)
    m.fp64_exp_eval.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_uint64, ctypes.c_void_p]
    rng = np.random.Generator(np.random.PCG64(8))
    kmax, kmin = float.fromhex("0x1.62e42fefa39efp+9"), float.fromhex("-0x1.74910d52d3052p+9")
    x = np.concatenate([np.linspace(kmin, kmax, 1_000_001), rng.uniform(-50, 50, 500_000),
                        rng.uniform(-745.2, -708.0, 200_000), np.array(
                            [0.0, -0.0, 1e-300, -1e-300, kmax, np.nextafter(kmax, 1e9), kmin,
                             np.nextafter(kmin, -1e9), -708.4, -1e10, 1e10, np.inf, -np.inf,
                             np.nan])])
    dx = torch.tensor(x, dtype=torch.float64, device="cuda")
    dy, dr = torch.empty_like(dx), torch.empty_like(dx)
    assert m.fp64_exp_eval(dx.data_ptr(), dy.data_ptr(), dr.data_ptr(), len(x),
                           torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    y, ref = dy.cpu().numpy(), dr.cpu().numpy()
    with np.errstate(over="ignore"):
        npref = np.exp(x)
    special = ~np.isfinite(npref) | (npref == 0) | np.isnan(x)
    assert np.array_equal(np.isnan(y), np.isnan(npref))
    assert np.array_equal(y[special & ~np.isnan(x)], npref[special & ~np.isnan(x)])
    ok = ~special
    for r in (ref[ok], npref[ok]):
        # distance in units in the last place (subnormals: units of 2^-1074)
        ulp = np.maximum(np.spacing(np.abs(r)), np.finfo(float).smallest_subnormal)
        assert np.max(np.abs(y[ok] - r) / ulp) <= 2.0
    assert y[np.where(x == 0.0)[0][0]] == 1.0


# ---------------------------------------------------------------- FP64 parity
def test_fp64_lepage_gauss_d4_run():
    """The d=4 Lepage Gaussian, 5 adapting iterations of 1e5 (a=0.1, 50 bins)."""
    wl = W.c1_gauss4()
    o = oracle.run(wl.dim, wl.nbins, wl.seed, wl.integrand, wl.params, wl.schedule, nthreads=8)
    g = gpu_run(wl.dim, wl.nbins, wl.seed, wl.integrand, wl.params, wl.schedule, V.VEGAS_FP64)
    assert_fp64_parity(g, o, wl.schedule)
    m, s, c, n, bad = g["result"]
    assert n == 5 and not bad
    assert rel(m, o["mean"]) < RTOL64 and rel(s, o["sigma"]) < 1e-10


def test_fp64_gauss_d8_adapt_then_fixed():
    """d=8 Gaussian: adapting then fixed-grid iterations (reduced sizes)."""
    sched = [(200_000, 1)] * 4 + [(500_001, 0)] * 2
    p = W.gauss_params(8, 0.1)
    o = oracle.run(8, 50, 2, W.GAUSS, p, sched, nthreads=8, first_iter=4)
    g = gpu_run(8, 50, 2, W.GAUSS, p, sched, V.VEGAS_FP64, first_iter=4)
    assert_fp64_parity(g, o, sched)
    m, s, c, n, bad = g["result"]
    assert n == 6 and rel(m, o["mean"]) < RTOL64 and rel(s, o["sigma"]) < 1e-10
    assert rel(c, o["chi2_dof"]) < 1e-8


@pytest.mark.parametrize("fid,dim,nbins", [(W.GAUSS_MIX2, 3, 37), (W.FLAT, 5, 7),
                                           (W.GENZ_DISC, 4, 20), (W.GENZ_PPEAK, 6, 25),
                                           (W.GAUSS, 1, 2), (W.GAUSS, 16, 100),
                                           (W.GAUSS, 2, 1024), (W.GAUSS, 8, 1),
                                           (W.GAUSS, 20, 50), (W.GAUSS_MIX2, 20, 40),
                                           (W.GENZ_DISC, 17, 20), (W.GENZ_PPEAK, 19, 30),
                                           (W.GAUSS, 8, 1024), (W.GAUSS, 20, 409)])
def test_fp64_integrands_and_shapes(fid, dim, nbins):
    if fid in (W.GAUSS, ):
        p = W.gauss_params(dim, 0.2, np.linspace(0.3, 0.7, dim))
    elif fid == W.GAUSS_MIX2:
        p = W.mix2_params(dim, 0.15)
    elif fid == W.FLAT:
        p = []
    else:
        p = W.genz_params(dim, seed=dim, kind=fid)
    sched = [(30_011, 1), (20_000, 1), (12_345, 0)]
    edges = W.random_monotone_grid(dim, nbins, seed=dim + nbins, spread=0.8) if nbins > 1 else None
    o = oracle.run(dim, nbins, 17, fid, p, sched, edges=edges, nthreads=8)
    g = gpu_run(dim, nbins, 17, fid, p, sched, V.VEGAS_FP64, edges=edges)
    assert_fp64_parity(g, o, sched)


@pytest.mark.parametrize("n", [2, 3, 31, 33, 255, 257, 1000])
def test_fp64_tiny_and_ragged_n(n):
    p = W.gauss_params(3, 0.3, [0.2, 0.5, 0.8])
    sched = [(n, 1), (n, 0)]
    o = oracle.run(3, 10, 5, W.GAUSS, p, sched)
    g = gpu_run(3, 10, 5, W.GAUSS, p, sched, V.VEGAS_FP64)
    assert_fp64_parity(g, o, sched)


def test_fewer_than_two_samples_are_refused():
    v = V.Vegas(3, 10, 1, V.VEGAS_FP64, W.GAUSS, W.gauss_params(3, 0.2), max_iters=4)
    for n in (0, 1):
        with pytest.raises(V.VegasError) as e:
            v.iterate(n, 1)
        assert e.value.status == V.VEGAS_EINVAL
    v.iterate(2, 1)
    assert v.iterations().shape[0] == 1
    v.close()


def test_launch_configuration_and_chunking_do_not_change_results():
    """Counters are a function of the sample index only: any block size, grid
    size or chunking gives the same sums (up to summation order)."""
    p = W.gauss_params(5, 0.1)
    sched = [(300_007, 1), (300_007, 1), (123_457, 0)]
    base = gpu_run(5, 50, 3, W.GAUSS, p, sched, V.VEGAS_FP64)
    for cfg in [dict(block_threads=64), dict(block_threads=128, blocks_per_sm=1),
                dict(chunk_samples=77_777), dict(min_samples_per_thread=1000)]:
        g = gpu_run(5, 50, 3, W.GAUSS, p, sched, V.VEGAS_FP64, cfg=cfg)
        assert rel(g["rows"][:, 4], base["rows"][:, 4]) < 1e-13
        assert np.allclose(g["edges"], base["edges"], rtol=1e-13, atol=1e-16)


def test_autotuner_picks_a_candidate_that_keeps_results():
    p = W.gauss_params(6, 0.15)
    cfg, timings = V.binding.autotune(6, 40, V.VEGAS_FP32_EVAL, W.GAUSS, p, 400_000,
                                      blocks=(128, 256), blocks_per_sm=(0, 2),
                                      min_samples=(8,), reps=2)
    assert len(timings) == 4 and all(t > 0 for t in timings.values())
    assert (cfg["block_threads"], cfg["blocks_per_sm"], cfg["min_samples_per_thread"]) in timings
    sched = [(300_007, 1), (300_007, 0)]
    base = gpu_run(6, 40, 3, W.GAUSS, p, sched, V.VEGAS_FP64)
    tuned = gpu_run(6, 40, 3, W.GAUSS, p, sched, V.VEGAS_FP64, cfg=cfg)
    assert rel(tuned["rows"][:, 4], base["rows"][:, 4]) < 1e-13


@pytest.mark.parametrize("fid,dim,nbins", [(W.GAUSS_MIX2, 16, 100), (W.GAUSS, 20, 50),
                                            (W.GENZ_PPEAK, 12, 64)])
def test_big_block_adapting_shape_equals_the_default_shape(fid, dim, nbins):
    """Float adapting iterations whose 32 lane-owned histogram copies miss the
    default budget run as one 768-thread block per SM; forcing the default
    shape (blocks_per_sm set) gives the same sums and histogram up to float
    summation order, and the same samples (the counters)."""
    if fid == W.GAUSS_MIX2:
        p = W.mix2_params(dim, 0.1)
    elif fid == W.GAUSS:
        p = W.gauss_params(dim, 0.1)
    else:
        p = W.genz_params(dim, seed=dim, kind=fid)
    out = []
    for cfg in ({}, {"blocks_per_sm": 1}):
        v = V.Vegas(dim, nbins, 5, V.VEGAS_FP32_EVAL, fid, p, max_iters=4)
        v.config(**cfg)
        v.iterate(1_000_003, 1)
        out.append((v.iterations()[0], v.histogram()))
        v.close()
    (rb, hb), (rd, hd) = out
    assert rb[2] == rd[2] and rb[3] == rd[3]
    assert abs(rb[4] - rd[4]) <= 1e-6 * abs(rd[4])
    assert np.allclose(hb, hd, rtol=1e-5, atol=1e-30 * np.max(hd))


def test_running_records_combine_like_the_oracle():
    """Vegas.records(): per iteration its own estimate and the combination of
    iterations first .. t (vegas_result_range), which equals the oracle's
    combination of the same logged rows and, at the last row, vegas_result."""
    p = W.gauss_params(5, 0.15)
    v = V.Vegas(5, 40, 8, V.VEGAS_FP64, W.GAUSS, p, max_iters=8)
    v.run([(100_000, 1)] * 4 + [(200_000, 0)] * 3)
    rows, recs = v.iterations(), v.records(first_iter=2)
    assert [r["iter"] for r in recs] == list(range(2, 7))
    for r in recs:
        t = r["iter"]
        assert r["I"] == rows[t][4] and r["n"] == rows[t][2]
        assert r["device_ms"] > 0 and r["samples_per_s"] > 0
        om, osg, oc = oracle.combine(rows[2:t + 1, 4], rows[2:t + 1, 5])
        assert abs(r["mean_so_far"] - om) <= 1e-13 * abs(om)
        assert abs(r["sigma_so_far"] - osg) <= 1e-13 * osg
        assert abs(r["chi2_dof_so_far"] - oc) <= 1e-12 * max(oc, 1.0)
    assert recs[0]["chi2_dof_so_far"] == 0.0
    assert abs(recs[0]["sigma_so_far"] - recs[0]["sigma"]) <= 1e-15 * recs[0]["sigma"]
    assert recs[-1]["mean_so_far"] == v.result(2)[0]
    with pytest.raises(V.VegasError) as e:  # not logged
        V.binding.vegas_result_range(v.handle, 0, 8)
    assert e.value.status == V.VEGAS_EINVAL
    v.close()


def test_tuning_table_with_the_real_autotuner(tmp_path):
    """TuningTable over the GPU autotuner: the stored choice is one of the
    candidates, is reused from the file, and keeps results."""
    p = W.gauss_params(5, 0.15)
    path = str(tmp_path / "tuning.json")
    kw = dict(blocks=(128, 256), blocks_per_sm=(0,), min_samples=(8,), reps=1)
    cfg = V.binding.TuningTable(path).lookup(5, 30, V.VEGAS_FP64, W.GAUSS, p, 300_007, True,
                                             **kw)
    assert cfg["block_threads"] in (128, 256)
    again = V.binding.TuningTable(path, tuner=lambda *a, **k: pytest.fail("re-tuned"))
    assert again.lookup(5, 30, V.VEGAS_FP64, W.GAUSS, p, 300_007, True) == cfg
    sched = [(300_007, 1), (300_007, 0)]
    base = gpu_run(5, 30, 3, W.GAUSS, p, sched, V.VEGAS_FP64)
    tuned = gpu_run(5, 30, 3, W.GAUSS, p, sched, V.VEGAS_FP64, cfg=cfg)
    assert rel(tuned["rows"][:, 4], base["rows"][:, 4]) < 1e-13


def test_one_call_integrate_equals_the_state_run_and_the_closed_form():
    p = W.gauss_params(4, 0.1)
    m, s, c = V.binding.integrate(V.VEGAS_GAUSS, p, 4, n_iter=6, n_events=200_000,
                                  mode=V.VEGAS_FP64, seed=5)
    g = gpu_run(4, 50, 5, W.GAUSS, p, [(200_000, 1)] * 5 + [(200_000, 0)], V.VEGAS_FP64,
                first_iter=5)
    assert abs(m - g["result"][0]) <= 1e-13 * abs(m)
    assert abs(m - math.erf(5.0) ** 4) < 5 * s
    # f = 1 over a box of volume 12 on the fixed uniform grid: f J is the volume
    # (FP64: exact to rounding; FP32-eval's sigma has a floor near
    # I sqrt(eps_f / n), the float rounding of every (f J)^2 alike)
    box = [(0.0, 2.0), (1.0, 4.0), (-1.0, 1.0)]
    mb, sb, _ = V.binding.integrate(V.VEGAS_FLAT, [], 3, n_iter=2, n_events=10_000,
                                    adapt_iters=0, box=box, mode=V.VEGAS_FP64)
    assert abs(mb - 12.0) < 1e-13 * 12 and sb < 1e-12
    mf, sf, _ = V.binding.integrate(V.VEGAS_FLAT, [], 3, n_iter=2, n_events=10_000,
                                    adapt_iters=0, box=box)
    assert abs(mf - 12.0) < 1e-6 * 12 and sf < 12 * 4 * math.sqrt(2.0 ** -23 / 20_000)
    # adapting to a flat integrand follows the histogram's sampling noise, so
    # the grid moves and the later estimate is only statistically exact
    ma, sa, _ = V.binding.integrate(V.VEGAS_FLAT, [], 3, n_iter=3, n_events=10_000, box=box)
    assert abs(ma - 12.0) < 5 * sa


def test_iteration_device_times_match_cuda_events():
    """vegas_get_iteration_times: each iteration's device time is positive, no
    longer than the CUDA-event time around its launches and most of it; a
    chunked iteration is timed across its launches."""
    p = W.gauss_params(8, 0.1)
    v = V.Vegas(8, 50, 2, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=8)
    s = torch.cuda.current_stream()
    v.iterate(10_000_000, 1)  # warm-up
    v.refine(1.5)
    events = []
    for n, cfg in [(10_000_000, {}), (100_000_000, {}), (100_000_000, {"chunk_samples": 25_000_000})]:
        if cfg:
            v.config(**cfg)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        v.iterate(n, 0)
        e1.record(s)
        events.append((e0, e1))
    torch.cuda.synchronize()
    t_dev = v.iteration_times() * 1e-6  # ms
    v.close()
    assert len(t_dev) == 4 and np.all(t_dev > 0)
    for (e0, e1), td in zip(events, t_dev[1:]):
        te = e0.elapsed_time(e1)
        assert 0.5 * te <= td <= te * 1.02 + 0.005, (td, te)


def test_fp64_nonfinite_is_counted_and_reported():
    """A width of 1e-300 makes the Gaussian's prefactor overflow: every f J is
    non-finite, is left out of the sums and vegas_result reports it."""
    p = [1e-300, 0.5, 0.5]
    o = oracle.iterate(oracle.uniform_grid(2, 10), 1, 0, 1000, W.GAUSS, p, adapt=True)
    g = gpu_run(2, 10, 1, W.GAUSS, p, [(1000, 1)], V.VEGAS_FP64)
    assert g["rows"][0][3] == o["nonfinite"] == 1000
    assert g["rows"][0][0] == 0.0
    assert g["result"][4] is True


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_full_size_d8_workload_one_step_parity(mode):
    """The d=8 Gaussian workload at full size (10 adapting iterations of 1e7,
    then 5 fixed-grid iterations of 1e8) in the default launch configuration,
    the one bench.py times.  For sampled iterations the oracle recomputes the
    iteration on the grid the GPU used (same counters), and the refinement from
    the GPU's own histogram; each comparison is then one step, with the FP64
    bound 1e-12 or the float budget 1e-5 (d=8)."""
    import os

    wl = W.c2_gauss8()
    v = V.Vegas(wl.dim, wl.nbins, wl.seed, mode, wl.integrand, wl.params, max_iters=16)
    grids, hists = [], {}
    check = [0, 4, 9, 10, 14]
    for t, (n, adapt) in enumerate(wl.schedule):
        grids.append(v.grid())
        v.iterate(n, adapt)
        if adapt:
            if t in check:
                hists[t] = v.histogram()
            v.refine(1.5)
    grids.append(v.grid())
    rows = v.iterations()
    v.close()
    tol = RTOL64 if mode == V.VEGAS_FP64 else 1e-5
    nt = os.cpu_count() or 1
    for t in check:
        n, adapt = wl.schedule[t]
        o = oracle.iterate(grids[t], wl.seed, t, n, wl.integrand, wl.params, adapt, nthreads=nt)
        assert rows[t][2] == n and rows[t][3] == o["nonfinite"] == 0
        assert rel(rows[t][4], o["I"]) < tol, (t, rows[t][4], o["I"])
        assert abs(rows[t][5] - o["var"]) <= 10 * tol * (o["var"] + o["I"] ** 2 / n), t
        if adapt:
            if mode == V.VEGAS_FP64:
                assert np.allclose(hists[t], o["hist"], rtol=1e-11, atol=0), t
            else:
                # bin by bin, within the float budget of one (f J)^2 bin
                h = prescale_h(rows[t - 1][4] if t > 0 else None)
                rt, at = fp32_hist_tol(wl.integrand, wl.dim, wl.params, grids[t], n, h=h)
                assert_hist_close(hists[t], o["hist"], rt, at, f"iteration {t}")
            # the refinement of the GPU's histogram: FP64 on both sides
            assert np.allclose(grids[t + 1], oracle.refine(grids[t], hists[t], 1.5),
                               rtol=RTOL64, atol=1e-15), t


@pytest.mark.parametrize("dim,sched", [(4, [(100_000, 1)] * 5),
                                       (8, [(1_000_000, 1)] * 8 + [(10_000_000, 0)] * 2)])
def test_fp64_every_step_of_a_whole_run_at_1e12(dim, sched):
    """FP64, every iteration of a whole run (config 1, and the d=8 schedule at
    reduced sample counts), one step at a time: the oracle recomputes
    iteration t on the grid the GPU ran it on (I and var 1e-12, every bin of
    the histogram 1e-11) and refines the GPU's own histogram into the GPU's
    next grid (1e-12).  Chained over the run, this is the whole run at the FP64
    bound; only comparing two independent runs needs the wider bound of
    fp64_tol, because each refinement amplifies the previous steps' rounding
    differences."""
    p = W.gauss_params(dim, 0.1)
    v = V.Vegas(dim, 50, 3, V.VEGAS_FP64, W.GAUSS, p, max_iters=len(sched) + 1)
    grids, hists = [], {}
    for t, (n, adapt) in enumerate(sched):
        grids.append(v.grid())
        v.iterate(n, adapt)
        if adapt:
            hists[t] = v.histogram()
            v.refine(1.5)
    grids.append(v.grid())
    rows = v.iterations()
    v.close()
    for t, (n, adapt) in enumerate(sched):
        o = oracle.iterate(grids[t], 3, t, n, W.GAUSS, p, adapt, nthreads=8)
        assert rel(rows[t][4], o["I"]) < RTOL64, (t, rows[t][4], o["I"])
        assert rel(rows[t][5], o["var"]) < 1e-10, t
        if adapt:
            assert np.allclose(hists[t], o["hist"], rtol=1e-11, atol=0), t
            assert np.allclose(grids[t + 1], oracle.refine(grids[t], hists[t], 1.5),
                               rtol=RTOL64, atol=1e-15), t
        else:
            assert np.array_equal(grids[t + 1], grids[t]), t


def _range_sums(mode, wl, grid, t, begin, end):
    """{S1, S2, nonfinite} of samples [begin, end) of iteration t of wl on
    `grid`, from a state advanced to iteration t (vegas_iterate_range)."""
    from paper_2002_12921_b300.shard import GpuShardEngine

    v = V.Vegas(wl.dim, wl.nbins, wl.seed, mode, wl.integrand, wl.params, max_iters=t + 2)
    v.set_grid(grid)
    # fixed-grid iterations move the iteration counter to t; on this grid their
    # estimate also sets the float path's pre-scale close to the real one
    for _ in range(t):
        v.iterate(1_000_000, 0)
    eng = GpuShardEngine(v)
    eng.iterate_range(wl.schedule[t][0], begin, end, False)
    out = eng.export()[:3].cpu().numpy().copy()
    v.close()
    return out


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
@pytest.mark.parametrize("dim,adapt", [(8, False), (3, False), (8, True)])
@pytest.mark.parametrize("first", [2**32 - 1_000_000, V.VEGAS_MAX_SAMPLE_INDEX - 2**32 - 1_000_000,
                                   V.VEGAS_MAX_SAMPLE_INDEX - 2_000_000])
def test_sample_ranges_across_a_high_word_boundary(mode, dim, adapt, first):
    """Index ranges whose threads cross a multiple of 2^32 (where the sample
    loop starts a new run of one high word and recomputes the per-call Philox
    constants), the last such crossing below the index bound, and the range
    that ends at the bound: the fixed-grid kernels above d = 4 (runs counted
    in 32 bits), at d = 3 and adapting (the 64-bit loop).  The range's sums,
    and in FP64 its histogram, equal the oracle's over the same indices."""
    from paper_2002_12921_b300.shard import GpuShardEngine

    p = W.gauss_params(dim, 0.1, np.linspace(0.3, 0.7, dim))
    e = oracle.run(dim, 40, 99, W.GAUSS, p, [(100_000, 1)] * 3)["edges"]
    count, n_total = 2_000_000, first + 2_000_000
    v = V.Vegas(dim, 40, 6, mode, W.GAUSS, p, max_iters=2)
    v.set_grid(e)
    eng = GpuShardEngine(v)
    eng.iterate_range(n_total, first, first + count, adapt)
    got = eng.export().cpu().numpy().copy()
    v.close()
    o = oracle.iterate_range(e, 6, 0, first, count, W.GAUSS, p, adapt, nthreads=8)
    tol = RTOL64 if mode == V.VEGAS_FP64 else 1e-5
    assert got[2] == o["nonfinite"] == 0
    assert rel(got[0], o["S1"]) < tol, (got[0], o["S1"])
    assert rel(got[1], o["S2"]) < 2 * tol, (got[1], o["S2"])
    if adapt and mode == V.VEGAS_FP64:
        assert np.allclose(got[3:].reshape(dim, 40), o["hist"], rtol=1e-11, atol=0)


def test_sample_indices_beyond_the_bound_are_refused():
    """n_total above VEGAS_MAX_SAMPLE_INDEX (where a thread's next index could
    wrap around 2^64) is refused before anything is enqueued."""
    v = V.Vegas(3, 10, 1, V.VEGAS_FP32_EVAL, W.GAUSS, W.gauss_params(3, 0.1), max_iters=2)
    top = V.VEGAS_MAX_SAMPLE_INDEX
    assert V.lib().vegas_iterate_range(v.handle, top + 1, top - 10, top, 0) == V.VEGAS_EINVAL
    assert V.lib().vegas_iterate(v.handle, top + 1, 0) == V.VEGAS_EINVAL
    assert V.lib().vegas_iterate_range(v.handle, top, top - 10, top, 0) == V.VEGAS_OK
    v.close()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_full_size_d16_mixture_sampled_parity(mode):
    """The d=16 mixture at full size (iterations of 1e9 samples in 1e8-sample
    launches, as bench.py runs it): on the grid of the third iteration, two
    sampled index ranges, one in the middle (across a launch boundary) and one
    ending at the last sample, reproduce the oracle's partial sums over the
    same indices; and
    (FP64) the ten 1e8-sample chunks' sums add up to the full iteration's sum."""
    import os

    wl = W.c5_mix16()
    n, t = wl.schedule[0][0], 2
    v = V.Vegas(wl.dim, wl.nbins, wl.seed, mode, wl.integrand, wl.params, max_iters=8)
    v.config(chunk_samples=wl.chunk)
    grids = []
    for _ in range(t + 1):
        grids.append(v.grid())
        v.iterate(n, 1)
        v.refine(1.5)
    rows = v.iterations()
    v.close()
    assert rows[t][2] == n
    tol = RTOL64 if mode == V.VEGAS_FP64 else 3e-5
    nt = os.cpu_count() or 1
    for begin in (n // 2 - 1_000_000, n - 2_000_000):
        end = begin + 2_000_000
        got = _range_sums(mode, wl, grids[t], t, begin, end)
        o = oracle.iterate_range(grids[t], wl.seed, t, begin, end - begin, wl.integrand,
                                 wl.params, False, nthreads=nt)
        assert got[2] == o["nonfinite"] == 0
        assert rel(got[0], o["S1"]) < tol, (begin, got[0], o["S1"])
        assert rel(got[1], o["S2"]) < 2 * tol, (begin, got[1], o["S2"])
    if mode == V.VEGAS_FP64:
        parts = [_range_sums(mode, wl, grids[t], t, c, c + wl.chunk)[0]
                 for c in range(0, n, wl.chunk)]
        assert rel(sum(parts), rows[t][0]) < 1e-13


def test_d16_mixture_reduced_run_fp64_first_iterations_equal_oracle():
    """Config 5's shape (d=16 two-peak mixture, a = 0.1, 100 bins) at 5e5
    samples per adapting iteration: the first three iterations -- the uniform
    grid and two refinements -- equal the oracle's at the FP64 bound
    (estimates, variances, histograms and grids)."""
    p = W.mix2_params(16, 0.1)
    sched = [(500_000, 1)] * 3
    o = oracle.run(16, 100, 5, W.GAUSS_MIX2, p, sched, nthreads=8)
    g = gpu_run(16, 100, 5, W.GAUSS_MIX2, p, sched, V.VEGAS_FP64)
    assert_fp64_parity(g, o, sched)


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_d16_mixture_reduced_run_locks_onto_one_peak_like_the_oracle(mode):
    """The same reduced run over 15 adapting iterations: the grid locks onto
    one diagonal peak in every dimension (>= 75 of 100 bins within 0.1 of its
    centre, <= 3 near the other) and the estimate combined over the last 5
    iterations is within 4 sigma of half the integral, as the oracle's does
    (tests/test_oracle_iterate.py); in FP64 it is the oracle's peak and the
    oracle's combined estimate to a hundredth of sigma (same counters; the
    rounding-level differences of each refinement grow over 15 of them: on
    the oracle itself, relative perturbations of 1e-15 per histogram bin move
    this combined estimate by 3e-4 sigma)."""
    from scipy.special import erf as erf_

    p = W.mix2_params(16, 0.1)
    sched = [(500_000, 1)] * 15
    g = gpu_run(16, 100, 5, W.GAUSS_MIX2, p, sched, mode, first_iter=10)
    J = 0.5 * (erf_((1 - 1 / 3) / 0.1) + erf_((1 / 3) / 0.1))
    half = 0.5 * J ** 16
    e = g["edges"]
    mids = 0.5 * (e[:, 1:] + e[:, :-1])
    near = np.stack([(np.abs(mids - c) < 0.1).sum(axis=1) for c in (1 / 3, 2 / 3)])
    won = int(np.argmax(near.sum(axis=1)))
    assert np.all(near[won] >= 75) and np.all(near[1 - won] <= 3), near
    m, sg = g["result"][0], g["result"][1]
    assert abs(m - half) < 4 * sg, (m, sg, half)
    if mode == V.VEGAS_FP64:
        o = oracle.run(16, 100, 5, W.GAUSS_MIX2, p, sched, nthreads=8, first_iter=10)
        oe = o["edges"]
        omids = 0.5 * (oe[:, 1:] + oe[:, :-1])
        assert int(np.argmax([(np.abs(omids - c) < 0.1).sum() for c in (1 / 3, 2 / 3)])) == won
        assert abs(m - o["mean"]) < 1e-2 * o["sigma"], (m, o["mean"], o["sigma"])


# ---------------------------------------------------------------- FP32-eval mode
def fp32_copies(dim, nbins):
    """(shared histogram copies, block threads) of a float adapting launch in
    the default configuration: 32 lane-owned copies in 256-thread blocks where
    they fit 52 KB, else one 768-thread block per SM with 32 copies where they
    fit its shared memory (d N up to ~1700 bins), else fewer copies."""
    if dim * nbins * 4 * 32 <= 52 * 1024:
        return 32, 256
    if dim * nbins * (8 + 4 * 32) <= 226 * 1024:
        return 32, 768
    lr = 5
    while lr > 0 and dim * nbins * 4 << lr > 52 * 1024:
        lr -= 1
    return 1 << lr, 256


@pytest.mark.parametrize("fid,dim,nbins,tol", [(W.GAUSS, 4, 50, 1e-5), (W.GAUSS, 8, 50, 1e-5),
                                               (W.GAUSS_MIX2, 16, 100, 3e-5),
                                               (W.GENZ_PPEAK, 6, 30, 1e-5),
                                               (W.GENZ_DISC, 5, 30, 1e-5), (W.FLAT, 3, 11, 1e-6),
                                               (W.GAUSS, 20, 50, 4e-5),
                                               (W.GAUSS, 8, 1024, 1e-5)])
def test_fp32_single_iteration_against_fp64_oracle(fid, dim, nbins, tol):
    """Same grid and counters: the float path's I and var are within the float
    error budget of the FP64 oracle's, and so is every bin of its (f J)^2
    histogram (the lane-owned float copies, their grouped compare-and-swap
    adds and the flush).  The d=16 mixture at N=100 and the d=20 Gaussian run
    the big-block shape (one 768-thread block per SM, 32 copies); d=8 at
    N=1024 runs with a single shared copy, where every add of a warp contends
    and the plain atomic add takes the lost races."""
    if fid == W.GAUSS:
        p = W.gauss_params(dim, 0.1)
    elif fid == W.GAUSS_MIX2:
        p = W.mix2_params(dim, 0.1)
    elif fid == W.FLAT:
        p = []
    else:
        p = W.genz_params(dim, seed=2 * dim, kind=fid)
    warm = oracle.run(dim, nbins, 99, fid, p, [(100_000, 1)] * 4, nthreads=8)
    e = warm["edges"]
    o = oracle.iterate(e, 7, 0, 400_000, fid, p, adapt=True, nthreads=8)
    g = gpu_run(dim, nbins, 7, fid, p, [(400_000, 1)], V.VEGAS_FP32_EVAL, edges=e)
    row = g["rows"][0]
    assert abs(row[4] - o["I"]) <= tol * abs(o["I"]) + 1e-300
    # a per-sample relative error delta of f J moves S2/n - I^2 by about
    # 2 delta (var n + I^2), so var moves by 2 delta (var + I^2/n)
    assert abs(row[5] - o["var"]) <= 10 * tol * (o["var"] + o["I"] ** 2 / 400_000)
    copies, block = fp32_copies(dim, nbins)
    rt, at = fp32_hist_tol(fid, dim, p, e, 400_000, copies=copies, block=block)
    assert_hist_close(g["hists"][0], o["hist"], rt, at, f"fid {fid} d {dim} N {nbins}")


def test_fp32_lepage_gauss_d4_within_3_sigma():
    wl = W.c1_gauss4()
    g = gpu_run(wl.dim, wl.nbins, wl.seed, wl.integrand, wl.params, wl.schedule,
                V.VEGAS_FP32_EVAL)
    o = oracle.run(wl.dim, wl.nbins, wl.seed, wl.integrand, wl.params, wl.schedule, nthreads=8)
    m, s, c, n, bad = g["result"]
    assert abs(m - o["mean"]) < 3 * np.hypot(s, o["sigma"]) / np.sqrt(2) + 1e-12 or \
        abs(m - o["mean"]) < 1e-4 * abs(o["mean"])
    assert abs(m - erf(5.0) ** 4) < 4 * s


def test_fp32_gauss_d8_close_to_fp64_gpu():
    """Same counters: the float and double runs differ by far less than their
    Monte Carlo error, and their errors agree to 1%."""
    sched = [(1_000_000, 1)] * 6 + [(2_000_000, 0)] * 2
    p = W.gauss_params(8, 0.1)
    g32 = gpu_run(8, 50, 2, W.GAUSS, p, sched, V.VEGAS_FP32_EVAL, first_iter=6)
    g64 = gpu_run(8, 50, 2, W.GAUSS, p, sched, V.VEGAS_FP64, first_iter=6)
    m32, s32 = g32["result"][:2]
    m64, s64 = g64["result"][:2]
    assert abs(m32 - m64) < 0.1 * s64
    assert abs(s32 / s64 - 1.0) < 0.01
    assert abs(m64 - erf(5.0) ** 8) < 4 * s64
    assert np.allclose(g32["edges"], g64["edges"], rtol=0, atol=1e-3)


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
@pytest.mark.parametrize("fid", [W.GENZ_DISC, W.GENZ_PPEAK])
def test_genz_16d_runs_reach_one(mode, fid):
    """Table 1's 16-dimensional Genz rows (Eq. 2 and Eq. 3, normalised to
    integrate to 1), with seeded parameters: 10 adapting iterations of 1e6 and
    5 fixed-grid iterations of 1e7 combine to 1 within 5 sigma, sigma < 1e-3."""
    p = W.genz_params(16, seed=16, kind=fid)
    v = V.Vegas(16, 50, 16, mode, fid, p, max_iters=16)
    v.run([(1_000_000, 1)] * 10 + [(10_000_000, 0)] * 5)
    mean, sigma, chi2, k, bad = v.result(10)
    v.close()
    assert k == 15 and not bad
    assert sigma < 1e-3, sigma
    assert abs(mean - 1.0) < 5 * sigma, (mean, sigma)


@pytest.mark.parametrize("fid", [W.GENZ_DISC, W.GENZ_PPEAK])
def test_genz_pulls_over_seeds_are_standard_normal(fid):
    """16-d Genz on a frozen adapted grid (FP32): (I - 1)/sigma over 200 seeds
    has mean ~0 and standard deviation ~1 (3-sigma bands)."""
    p = W.genz_params(16, seed=16, kind=fid)
    warm = V.Vegas(16, 50, 16, V.VEGAS_FP64, fid, p, max_iters=8)
    warm.run([(1_000_000, 1)] * 6)
    grid = warm.grid()
    warm.close()
    pulls = []
    for seed in range(200):
        v = V.Vegas(16, 50, 5000 + seed, V.VEGAS_FP32_EVAL, fid, p, max_iters=2)
        v.set_grid(grid)
        v.iterate(200_000, 0)
        row = v.iterations()[0]
        v.close()
        pulls.append((row[4] - 1.0) / np.sqrt(row[5]))
    pulls = np.array(pulls)
    assert abs(pulls.mean()) < 3 / np.sqrt(200)
    assert abs(pulls.std() - 1) < 3 / np.sqrt(2 * 200)


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_pulls_over_seeds_are_standard_normal(mode):
    """On a frozen adapted grid, (I - I_exact)/sigma over 200 seeds has mean ~0
    and standard deviation ~1 (3-sigma bands of the sample moments)."""
    dim, a = 4, 0.1
    p = W.gauss_params(dim, a)
    warm = V.Vegas(dim, 50, 999, V.VEGAS_FP64, W.GAUSS, p, max_iters=8)
    warm.run([(200_000, 1)] * 6)
    grid = warm.grid()
    warm.close()
    exact = float(erf(0.5 / a) ** dim)
    pulls = []
    for seed in range(200):
        v = V.Vegas(dim, 50, seed, mode, W.GAUSS, p, max_iters=2)
        v.set_grid(grid)
        v.iterate(20_000, 0)
        row = v.iterations()[0]
        v.close()
        pulls.append((row[4] - exact) / np.sqrt(row[5]))
    pulls = np.array(pulls)
    assert abs(pulls.mean()) < 3 / np.sqrt(200)
    assert abs(pulls.std() - 1) < 3 / np.sqrt(2 * 200)


@pytest.mark.parametrize("fid,dim", [(W.GAUSS, 8), (W.GAUSS, 3), (W.GAUSS, 1), (W.GAUSS, 4),
                                     (W.GENZ_PPEAK, 6), (W.GENZ_PPEAK, 2), (W.GENZ_DISC, 8),
                                     (W.GENZ_DISC, 5), (W.GAUSS_MIX2, 5), (W.GAUSS_MIX2, 7),
                                     (W.FLAT, 1), (W.FLAT, 8), (W.GAUSS, 16), (W.GENZ_DISC, 12),
                                     (W.GAUSS_MIX2, 9), (W.GAUSS, 17)])
def test_fixed_grid_kernel_compiled_for_50_bins_equals_the_general_one(fid, dim):
    """Float fixed-grid iterations at 50 bins (up to d = 16; d = 17 takes the
    general kernel either way) run, under the
    default launch configuration, a kernel with the bin count compiled in; the
    general kernel (taken under an explicit blocks-per-SM setting) gives the
    same sums up to their order of summation, and both equal the oracle's
    within the float budget."""
    if fid == W.GAUSS:
        p = W.gauss_params(dim, 0.1)
    elif fid == W.GAUSS_MIX2:
        p = W.mix2_params(dim, 0.15)
    elif fid == W.FLAT:
        p = []
    else:
        p = W.genz_params(dim, seed=dim, kind=fid)
    e = oracle.run(dim, 50, 9, fid, p, [(100_000, 1)] * 3)["edges"]
    rows = []
    # default (compiled kernel), the general kernel, the compiled kernel chunked
    for cfg in ({}, {"blocks_per_sm": 4}, {"chunk_samples": 7_000_003}):
        v = V.Vegas(dim, 50, 9, V.VEGAS_FP32_EVAL, fid, p, max_iters=2)
        v.set_grid(e)
        if cfg:
            v.config(**cfg)
        v.iterate(20_000_000, 0)
        rows.append(v.iterations()[0])
        v.close()
    o = oracle.iterate(e, 9, 0, 20_000_000, fid, p, False, nthreads=8)
    for r in rows:
        assert r[2] == 20_000_000 and r[3] == o["nonfinite"] == 0
        assert rel(r[4], o["I"]) < 1e-5, (r[4], o["I"])
    for r in rows[1:]:
        assert rel(rows[0][0], r[0]) < 1e-7 and rel(rows[0][1], r[1]) < 1e-7
