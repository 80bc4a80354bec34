"""The batched persistent launch (vegas_batch_*) against the oracle, integral
by integral: integral b of a batch must reproduce a single run with integral
id b in the Philox counter."""
import numpy as np
import pytest
from scipy.special import erf

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


def small_batch():
    """Six Gaussians of uneven dimension (up to the maximum, 20) and sample
    count."""
    rng = np.random.Generator(np.random.PCG64(11))
    dims = [2, 5, 8, 13, 16, 20]
    ns = [3000, 20011, 12345, 7777, 40000, 15001]
    params = [W.gauss_params(d, float(rng.uniform(0.1, 0.3)), rng.uniform(0.3, 0.7, d))
              for d in dims]
    return dims, ns, params


def closed(p):
    a, mu = p[0], np.asarray(p[1:])
    return float(np.prod(0.5 * (erf((1 - mu) / a) + erf(mu / a))))


def fp64_tol(edges):
    dmin = np.min(np.diff(edges, axis=1))
    return max(1e-12, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def test_batch_fp64_matches_single_integral_oracle_runs():
    dims, ns, params = small_batch()
    sched_adapt, iters = 3, 4  # three adapting iterations, then one on the frozen grid
    B = V.VegasBatch(dims, ns, 30, 7, V.VEGAS_FP64, params, max_iters=8)
    B.config(tile_samples=4096)
    B.reset()
    for t in range(iters):
        B.iterate(adapt=t < sched_adapt)
    log = B.log()
    for b, (d, n, p) in enumerate(zip(dims, ns, params)):
        o = oracle.run(d, 30, 7, W.GAUSS, p, [(n, 1)] * sched_adapt + [(n, 0)],
                       integral_id=b, nthreads=4)
        for t in range(iters):
            tol = 1e-12 if t == 0 else fp64_tol(o["grids"][t])
            assert log[b, t, 2] == n
            assert abs(log[b, t, 4] - o["log"][t]["I"]) <= tol * abs(o["log"][t]["I"]), (b, t)
            assert abs(log[b, t, 5] - o["log"][t]["var"]) <= 100 * tol * o["log"][t]["var"]
        assert np.allclose(B.grid(b), o["edges"], rtol=1e-12, atol=1e-15)
        # the histogram the last refinement used (iteration 2), bin by bin
        htol = max(1e-11, 2 * fp64_tol(o["grids"][2]))
        assert np.allclose(B.histogram(b), o["log"][2]["hist"], rtol=htol, atol=0), b
        m, s, c, k, bad = B.result(b)
        assert k == iters and not bad
    B.close()


@pytest.mark.parametrize("tile", [0, 4096])
def test_batch_fp32_histograms_bin_by_bin_against_the_oracle(tile):
    """FP32 tiles of the persistent kernel: the (f J)^2 histogram each
    integral's first refinement used (uniform grid, same counters) equals the
    oracle's bin by bin within the float budget of one bin, and the refined
    grid equals the oracle's refinement of its own histogram within what that
    budget lets a refinement move.  The widest integral (d = 20 at N = 30, 600
    bins) misses the default 52 KB budget for 32 copies, so the round runs as
    one 768-thread block per SM, every tile with lane-owned copies; tile 4096
    spreads one integral's samples over many tiles, each flushed on its own."""
    from tests.fp32_budget import assert_hist_close, fp32_hist_tol, refine_edge_tol

    dims, ns, params = small_batch()
    B = V.VegasBatch(dims, ns, 30, 7, V.VEGAS_FP32_EVAL, params, max_iters=4)
    if tile:
        B.config(tile_samples=tile)
    B.reset()
    B.iterate(adapt=True)
    for b, (d, n, p) in enumerate(zip(dims, ns, params)):
        e = oracle.uniform_grid(d, 30)
        o = oracle.iterate(e, 7, 0, n, W.GAUSS, p, True, integral_id=b, nthreads=4)
        rt, at = fp32_hist_tol(W.GAUSS, d, p, e, min(n, tile or 65536), copies=32, sms=1,
                               block=768)
        assert_hist_close(B.histogram(b), o["hist"], rt, at, f"integral {b} (d={d})")
        etol = refine_edge_tol(e, o["hist"], 1.5, rt)
        assert np.allclose(B.grid(b), oracle.refine(e, o["hist"], 1.5), rtol=0, atol=etol), b
    B.close()


def test_tile_size_and_block_size_do_not_change_results():
    dims, ns, params = small_batch()
    runs = []
    for bt, ts in [(256, 4096), (128, 65536), (64, 8192)]:
        B = V.VegasBatch(dims, ns, 30, 9, V.VEGAS_FP64, params, max_iters=4)
        B.config(block_threads=bt, tile_samples=ts)
        B.run(3)
        grids = np.concatenate([B.grid(b).ravel() for b in range(len(dims))])
        runs.append((B.log()[:, :3, 4], grids))
        B.close()
    for I, e in runs[1:]:
        assert np.allclose(I, runs[0][0], rtol=1e-12, atol=0)
        assert np.allclose(e, runs[0][1], rtol=1e-12, atol=1e-15)


def test_batch_fp32_close_to_fp64():
    dims, ns, params = small_batch()
    out = {}
    for mode in (V.VEGAS_FP64, V.VEGAS_FP32_EVAL):
        B = V.VegasBatch(dims, ns, 30, 5, mode, params, max_iters=4)
        B.run(4)
        out[mode] = [B.result(b, 1) for b in range(len(dims))]
        B.close()
    for r64, r32 in zip(out[V.VEGAS_FP64], out[V.VEGAS_FP32_EVAL]):
        assert abs(r32[0] - r64[0]) < 0.05 * r64[1]
        assert abs(r32[1] / r64[1] - 1) < 0.01


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_graph_replay_equals_eager_run(mode):
    """A replayed graph reruns the same iterations.  The runs differ only in
    the order of atomic additions: FP64 agrees to 1e-9 over six refinements.
    In FP32 the shared histogram's float atomics from different warps land in
    a run-dependent order and the refinements amplify that on the hard d=16
    integral, so only the first (uniform-grid) iteration is compared there,
    to 1e-6."""
    dims, ns, params = small_batch()
    B = V.VegasBatch(dims, ns, 30, 13, mode, params, max_iters=8)
    B.run(6)
    eager = B.log()
    graph = B.capture(6)
    upto = 6 if mode == V.VEGAS_FP64 else 1
    rtol = 1e-9 if mode == V.VEGAS_FP64 else 1e-6
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        replay = B.log()
        assert np.array_equal(replay[:, :6, 2], eager[:, :6, 2])
        assert np.allclose(replay[:, :upto, 4], eager[:, :upto, 4], rtol=rtol, atol=0)
        assert B.result(3)[3] == 6
    B.close()


def test_autotuner_picks_a_candidate_and_keeps_results():
    """The autotuner's space: block sizes 128, 256 and 512, samples per thread
    (tile = block x s) from 1 up; whichever it picks, and any candidate forced,
    the results are those of the default configuration (FP64, 1e-12)."""
    dims, ns, params = small_batch()
    B = V.VegasBatch(dims, ns, 30, 17, V.VEGAS_FP64, params, max_iters=4)
    (bt, ts, by_dim), timings = V.binding.autotune_batch(
        B, blocks=(128, 256, 512), samples_per_thread=(1, 16, 256), reps=1)
    assert (bt, ts) in timings and len(timings) >= 9
    assert {(512, 512), (128, 128), (256, 65536)} <= set(timings)
    assert all(d in dims and t >= 128 for d, t in by_dim.items())
    B.run(2)
    tuned = B.log()[:, :2, 4]
    for cfg in ((256, 65536), (512, 512), (128, 128)):
        B.config(block_threads=cfg[0], tile_samples=cfg[1])
        B.config_tiles_by_dim({})
        B.run(2)
        assert np.allclose(B.log()[:, :2, 4], tuned, rtol=1e-12), cfg
    B.close()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_tuning_table_configures_a_batch_without_changing_results(mode, tmp_path):
    """TuningTable.lookup_batch tunes a batch (512-thread blocks included),
    keeps its choice per dimension bucket and configures a second batch of
    the same key from the file; both give the default configuration's
    results (FP64 1e-12; FP32 the first, uniform-grid iteration to 1e-6, the
    float histogram's atomics landing in another order afterwards)."""
    dims, ns, params = small_batch()
    ref = V.VegasBatch(dims, ns, 30, 23, mode, params, max_iters=3)
    ref.run(2)
    expect = ref.log()[:, :2, 4]
    ref.close()
    path = str(tmp_path / "tuning.json")
    for _ in range(2):
        B = V.VegasBatch(dims, ns, 30, 23, mode, params, max_iters=3)
        e = V.binding.TuningTable(path).lookup_batch(
            B, blocks=(256, 512), samples_per_thread=(16, 256), reps=1)
        assert e["block_threads"] in (256, 512)
        B.run(2)
        got = B.log()[:, :2, 4]
        B.close()
        if mode == V.VEGAS_FP64:
            assert np.allclose(got, expect, rtol=1e-12)
        else:
            assert np.allclose(got[:, 0], expect[:, 0], rtol=1e-6)


def test_tiles_by_dimension_do_not_change_results():
    dims, ns, params = small_batch()
    logs = []
    for by_dim in ({}, {2: 4096, 8: 65536, 16: 8192, 20: 4096}):
        B = V.VegasBatch(dims, ns, 30, 19, V.VEGAS_FP64, params, max_iters=4)
        B.config_tiles_by_dim(by_dim)
        B.run(3)
        logs.append((B.log()[:, :3, 4], np.concatenate([B.grid(b).ravel()
                                                        for b in range(len(dims))])))
        B.close()
    assert np.allclose(logs[1][0], logs[0][0], rtol=1e-12, atol=0)
    assert np.allclose(logs[1][1], logs[0][1], rtol=1e-12, atol=1e-15)
    with pytest.raises(V.VegasError):
        B = V.VegasBatch(dims, ns, 30, 19, V.VEGAS_FP64, params, max_iters=4)
        try:
            B.config_tiles_by_dim({3: 100})  # below the 128 minimum
        finally:
            B.close()


def _combine(I, var):
    w = 1.0 / var
    return float(np.sum(I * w) / np.sum(w)), float(np.sum(w) ** -0.5)


def test_full_batch_of_256():
    """The 256-integral workload (d ~ U{2..16}, n log-uniform in [1e4, 1e6],
    a ~ U(0.05, 0.3), centres ~ U(0.2, 0.8), 50 bins, 8 adapting iterations),
    replayed from a CUDA graph.
    FP64, against the oracle on every 16th integral: each of iterations 0..3
    within the per-refinement bound (max(1e-12, 8 d eps / min Delta) of the
    grid it ran on), and the result combined over iterations 3..7 within a
    thousandth of its Monte Carlo error.  (Each refinement amplifies the
    previous grids' one-ulp differences, so on the hardest d=16 integrals later
    iterations drift past the one-step bound, to ~1e-7 relative after eight.)
    FP32: iteration 0 runs on the same uniform grid as FP64 and agrees to the
    d=16 float bound 3e-5 wherever the estimate is not float underflow
    (I > 1e-30); over whole runs FP32 finds as many integrals within 5 sigma
    of their closed form as FP64, less three (on the hardest integrals the
    first refinements see float-underflowed tails as zero and follow another
    valid grid trajectory)."""
    wls = W.c4_batch()
    dims = [w.dim for w in wls]
    ns = [w.schedule[0][0] for w in wls]
    params = [w.params for w in wls]
    logs = {}
    for mode in (V.VEGAS_FP64, V.VEGAS_FP32_EVAL):
        B = V.VegasBatch(dims, ns, 50, wls[0].seed, mode, params, max_iters=8)
        graph = B.capture(8)
        graph.replay()
        torch.cuda.synchronize()
        logs[mode] = B.log()
        B.close()
    g64, g32 = logs[V.VEGAS_FP64], logs[V.VEGAS_FP32_EVAL]
    for b in range(0, 256, 16):
        w = wls[b]
        o = oracle.run(w.dim, 50, w.seed, W.GAUSS, w.params, w.schedule, integral_id=b,
                       nthreads=8)
        for t in range(4):
            tol = 1e-12 if t == 0 else fp64_tol(o["grids"][t])
            ref = o["log"][t]["I"]
            assert abs(g64[b, t, 4] - ref) <= tol * abs(ref), (b, t)
        m_o, s_o = _combine(np.array([r["I"] for r in o["log"][3:]]),
                            np.array([r["var"] for r in o["log"][3:]]))
        m_g, _ = _combine(g64[b, 3:, 4], g64[b, 3:, 5])
        assert abs(m_g - m_o) <= 1e-3 * s_o, b
    ok = g64[:, 0, 4] > 1e-30
    assert np.all(np.abs(g32[ok, 0, 4] - g64[ok, 0, 4]) <= 3e-5 * g64[ok, 0, 4])
    within = {}
    for mode, g in ((V.VEGAS_FP64, g64), (V.VEGAS_FP32_EVAL, g32)):
        within[mode] = sum(abs(_combine(g[b, 3:, 4], g[b, 3:, 5])[0] - closed(p)) <
                           5 * _combine(g[b, 3:, 4], g[b, 3:, 5])[1]
                           for b, p in enumerate(params))
    assert within[V.VEGAS_FP64] >= 230
    assert within[V.VEGAS_FP32_EVAL] >= within[V.VEGAS_FP64] - 3


# ------------------------------------------- other integrands and boxes
def family_batch(fid):
    """Four integrals of one family, uneven dimension and sample count; the
    second and fourth over boxes (the rest on the unit cube)."""
    dims = [2, 5, 3, 7]
    ns = [20_011, 15_000, 9_999, 12_000]
    if fid == W.GAUSS_MIX2:
        params = [W.mix2_params(d, 0.2) for d in dims]
    elif fid == W.FLAT:
        params = [[] for _ in dims]
    else:
        params = [W.genz_params(d, seed=10 + d, kind=fid) for d in dims]
    boxes = [None, [(-1.0, 2.0)] * 5, None, [(0.25 * k, 0.25 * k + 1.5) for k in range(7)]]
    return dims, ns, params, boxes


@pytest.mark.parametrize("fid", [W.GAUSS_MIX2, W.FLAT, W.GENZ_DISC, W.GENZ_PPEAK])
def test_batch_of_any_builtin_integrand_matches_the_oracle(fid):
    """FP64: every integral of a batch of the family equals the oracle's run
    with its integral id and box, iteration by iteration, and its final grid."""
    dims, ns, params, boxes = family_batch(fid)
    B = V.VegasBatch(dims, ns, 25, 17, V.VEGAS_FP64, params, max_iters=6, integrand=fid,
                     boxes=boxes)
    B.config(tile_samples=4096)
    B.reset()
    for t in range(4):
        B.iterate(adapt=t < 3)
    log = B.log()
    for b, (d, n, p, box) in enumerate(zip(dims, ns, params, boxes)):
        o = oracle.run(d, 25, 17, fid, p, [(n, 1)] * 3 + [(n, 0)], integral_id=b, nthreads=4,
                       box=box)
        for t in range(4):
            tol = 1e-12 if t == 0 else fp64_tol(o["grids"][t])
            I = o["log"][t]["I"]
            assert log[b, t, 2] == n
            assert abs(log[b, t, 4] - I) <= tol * abs(I) + 1e-300, (fid, b, t, log[b, t, 4], I)
        assert np.allclose(B.grid(b), o["edges"], rtol=max(1e-12, 2 * fp64_tol(o["grids"][2])),
                           atol=1e-15)
    B.close()


def test_fp32_boxed_mixture_batch_first_iteration_within_float_bound():
    dims, ns, params, boxes = family_batch(W.GAUSS_MIX2)
    B = V.VegasBatch(dims, ns, 25, 17, V.VEGAS_FP32_EVAL, params, max_iters=4,
                     integrand=W.GAUSS_MIX2, boxes=boxes)
    B.reset()
    B.iterate(adapt=True)
    log = B.log()
    for b, (d, n, p, box) in enumerate(zip(dims, ns, params, boxes)):
        o = oracle.iterate(oracle.uniform_grid(d, 25), 17, 0, n, W.GAUSS_MIX2, p, True,
                           integral_id=b, box=box)
        assert abs(log[b, 0, 4] - o["I"]) <= 1e-5 * abs(o["I"]), b
    B.close()


def test_batch_init_refuses_bad_integrands_and_boxes():
    dims, ns = [2, 3], [5000, 5000]
    with pytest.raises(V.VegasError) as e:  # no caller-compiled integrands in a batch
        V.VegasBatch(dims, ns, 10, 1, V.VEGAS_FP64, [[], []], integrand=V.VEGAS_USER)
    assert e.value.status == V.VEGAS_EINVAL
    with pytest.raises(V.VegasError) as e:  # an empty interval
        V.VegasBatch(dims, ns, 10, 1, V.VEGAS_FP64, [[], []], integrand=W.FLAT,
                     boxes=[None, [(0.0, 1.0), (1.0, 1.0), (0.0, 1.0)]])
    assert e.value.status == V.VEGAS_EINVAL


def test_big_block_batch_round_equals_the_default_shape():
    """Float adapting rounds whose 32 copies for the widest integral miss the
    default budget run as one 768-thread block per SM; forcing the default
    shape (128-thread blocks) gives the same samples, sums to float summation
    order and the same refined grids to float rounding."""
    dims, ns, params = small_batch()  # widest: d = 20 at N = 30, 600 bins
    out = []
    for bt in (256, 128):
        B = V.VegasBatch(dims, ns, 30, 7, V.VEGAS_FP32_EVAL, params, max_iters=4)
        B.config(block_threads=bt, tile_samples=8192)
        B.run(1)
        out.append((B.log()[:, 0], [B.grid(b) for b in range(len(dims))]))
        B.close()
    (lb, gb), (ld, gd) = out
    assert np.array_equal(lb[:, 2:4], ld[:, 2:4])
    assert np.allclose(lb[:, 4], ld[:, 4], rtol=1e-6, atol=0)
    for b in range(len(dims)):
        assert np.allclose(gb[b], gd[b], rtol=0, atol=1e-6), b
