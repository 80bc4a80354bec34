"""Different states may be driven concurrently (include/vegas.h, Threads):
four states, each on its own stream and host thread, with different shapes,
integrands and precisions, run their schedules at the same time and reproduce
the same runs done one after another (up to summation order)."""
import threading

import numpy as np
import pytest

import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    (V.VEGAS_FP64, W.GAUSS, 6, 40, lambda: W.gauss_params(6, 0.15)),
    (V.VEGAS_FP32_EVAL, W.GAUSS, 8, 50, lambda: W.gauss_params(8, 0.1)),
    (V.VEGAS_FP32_EVAL, W.GAUSS_MIX2, 5, 30, lambda: W.mix2_params(5, 0.2)),
    (V.VEGAS_FP64, W.GENZ_PPEAK, 4, 25, lambda: W.genz_params(4, seed=4, kind=W.GENZ_PPEAK)),
]
SCHED = [(400_000, 1)] * 4 + [(1_000_003, 0)] * 2


def run_case(i, stream):
    mode, fid, dim, nbins, params = CASES[i]
    with torch.cuda.stream(stream):
        v = V.Vegas(dim, nbins, 100 + i, mode, fid, params(), max_iters=8, stream=stream)
        v.config(chunk_samples=300_000)
        v.run(SCHED)
        out = (v.iterations(), v.grid())
        v.close()
    return out


def test_concurrent_states_on_their_own_streams_and_threads():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()
    streams = [torch.cuda.Stream() for _ in CASES]
    sequential = [run_case(i, streams[i]) for i in range(len(CASES))]
    results, errors = [None] * len(CASES), []

    def worker(i):
        try:
            results[i] = run_case(i, streams[i])
        except Exception as exc:  # reported below
            errors.append((i, exc))

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(len(CASES))]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    for i, (mode, *_rest) in enumerate(CASES):
        rows, grid = results[i]
        ref_rows, ref_grid = sequential[i]
        tol = 1e-13 if mode == V.VEGAS_FP64 else 1e-5
        assert np.array_equal(rows[:, 2:4], ref_rows[:, 2:4]), i
        assert np.allclose(rows[:, 4], ref_rows[:, 4], rtol=tol, atol=0), i
        assert np.allclose(grid, ref_grid, rtol=0, atol=10 * tol), i


def test_states_sharing_a_kernel_with_different_shared_memory():
    """Two float states of one kernel (d=8 adapting, 32 histogram copies) with
    different bin counts need different dynamic shared memory (54.4 KB at 50
    bins, 43.5 KB at 40); each state prepares a launch shape once and keeps
    it.  Iterations interleaved between them run and equal each state's run
    on its own."""
    import paper_2002_12921_b300 as V
    from paper_2002_12921_b300 import workloads as W

    p = W.gauss_params(8, 0.1)
    alone = []
    for nbins in (50, 40):
        v = V.Vegas(8, nbins, 5, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=4)
        v.run([(1_000_000, 1)] * 3)
        alone.append(v.iterations())
        v.close()
    a = V.Vegas(8, 50, 5, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=4)
    b = V.Vegas(8, 40, 5, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=4)
    for _ in range(3):
        a.iterate(1_000_000, 1)
        b.iterate(1_000_000, 1)
        a.refine(1.5)
        b.refine(1.5)
    for v, ref in zip((a, b), alone):
        rows = v.iterations()
        v.close()
        assert np.array_equal(rows[:, 2], ref[:, 2])
        # the first iteration is on the uniform grid: the same sums to float order
        assert np.allclose(rows[0, 4], ref[0, 4], rtol=1e-6)
        assert np.allclose(rows[:, 4], ref[:, 4], rtol=1e-4)


def test_pinned_staging_reused_across_states_and_threads():
    """Destroyed states return their pinned log staging to the library's pool
    and new states take it (include/vegas.h, vegas_init_grid): four host
    threads each create, run, read and destroy 25 states of mixed log lengths
    (staging sizes of 32, 64 and 128 rows) on their own streams.  Every run's
    log equals the same run done alone, so no block was ever held by two
    states at once.  Fixed-grid iterations only, so the sums are
    deterministic and the logs compared bit for bit."""
    import paper_2002_12921_b300 as V
    from paper_2002_12921_b300 import workloads as W

    p = W.gauss_params(3, 0.2)
    lengths = (3, 20, 40, 70)

    def run(seed, max_iters, stream):
        with torch.cuda.stream(stream):
            v = V.Vegas(3, 16, seed, V.VEGAS_FP64, W.GAUSS, p, max_iters=max_iters,
                        stream=stream)
            v.run([(60_000 + 1000 * seed, 0)] * 3)
            rows = v.iterations()
            v.close()
        return rows

    streams = [torch.cuda.Stream() for _ in range(4)]
    ref = {(t, k): run(10 * t + k, lengths[(t + k) % 4], streams[t])
           for t in range(4) for k in range(5)}
    errors = []

    def worker(t):
        try:
            for c in range(25):
                k = c % 5
                rows = run(10 * t + k, lengths[(t + k) % 4], streams[t])
                if not np.array_equal(rows, ref[(t, k)]):
                    errors.append((t, c))
        except Exception as exc:  # reported below
            errors.append((t, exc))

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
    assert not errors, errors


def test_batches_sharing_a_kernel_with_different_shared_memory_on_threads():
    """Two float batches whose widest integral has d = 16, at 50 and 100 bins,
    launch the same big-block adapting kernel with different dynamic shared
    memory (102 KB and 205 KB of histogram copies).  Run concurrently from two
    host threads on their own streams, every round of each launches (the
    kernel's limit is raised once, to the device's maximum, and never lowered
    by the other batch) and reproduces the batch run alone: sample and
    non-finite counts exactly, the first round's sums (uniform grid) up to the
    order of the tiles' FP64 atomic adds, the later rounds within float
    rounding of the refined grids."""
    import paper_2002_12921_b300 as V
    from paper_2002_12921_b300 import workloads as W

    dims = [16, 5, 9]
    ns = [300_000, 120_000, 200_000]
    params = [W.gauss_params(d, 0.2) for d in dims]
    streams = [torch.cuda.Stream() for _ in range(2)]

    def run(nbins, stream):
        with torch.cuda.stream(stream):
            B = V.VegasBatch(dims, ns, nbins, 21, V.VEGAS_FP32_EVAL, params, max_iters=4,
                             stream=stream)
            B.run(4)
            out = B.log()
        return out

    alone = [run(nb, streams[i]) for i, nb in enumerate((50, 100))]
    results, errors = [None, None], []

    def worker(i, nbins):
        try:
            for _ in range(5):
                results[i] = run(nbins, streams[i])
        except Exception as exc:  # reported below
            errors.append((i, exc))

    threads = [threading.Thread(target=worker, args=(i, nb)) for i, nb in enumerate((50, 100))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
    assert not errors, errors
    for got, ref in zip(results, alone):
        assert np.array_equal(got[:, :, 2:4], ref[:, :, 2:4])
        assert np.allclose(got[:, 0, :2], ref[:, 0, :2], rtol=1e-12, atol=0)
        assert np.allclose(got[:, :, 4], ref[:, :, 4], rtol=1e-4, atol=0)


def test_pinned_pool_overflow_frees_the_surplus():
    """More live states than the pinned pool keeps (64): 80 states created,
    iterated and read, then all destroyed (the pool keeps 64 blocks and frees
    the other 16), then 80 more created from the refilled pool; every log
    equals a lone run's."""
    import paper_2002_12921_b300 as V
    from paper_2002_12921_b300 import workloads as W

    p = W.gauss_params(2, 0.3)

    def make(seed):
        v = V.Vegas(2, 8, seed, V.VEGAS_FP64, W.GAUSS, p, max_iters=3)
        v.iterate(20_000, 0)
        return v

    ref = make(0)
    want = ref.iterations()
    ref.close()
    for _ in range(2):
        states = [make(0) for _ in range(80)]
        for v in states:
            assert np.array_equal(v.iterations(), want)
        for v in states:
            v.close()


def test_log_longer_than_the_pinned_staging_is_read_in_pieces():
    """A log of 4500 rows, longer than the 4096 rows a state's pinned staging
    holds, is read back through it in pieces (vegas_get_iterations and
    vegas_result); the rows equal the log copied straight from the device by
    vegas_export_state (blob: 16 header words, the parameters, grid,
    histogram, then 8 doubles per row), and the combined result equals the
    combination of those rows."""
    import struct

    import oracle
    import paper_2002_12921_b300 as V
    from paper_2002_12921_b300 import workloads as W

    dim, nbins, iters, n = 2, 8, 4500, 1000
    p = W.gauss_params(dim, 0.3)
    v = V.Vegas(dim, nbins, 3, V.VEGAS_FP64, W.GAUSS, p, max_iters=iters)
    for _ in range(iters):
        v.iterate(n, 0)
    rows = v.iterations()
    mean, sigma, chi2, n_iter, _ = v.result(0)
    blob = v.export_state()
    v.close()
    (np_,) = struct.unpack_from("<Q", blob, 56)
    off = 8 * (16 + np_ + dim * (nbins + 1) + dim * nbins)
    log = np.frombuffer(blob, dtype="<f8", count=iters * 8, offset=off).reshape(iters, 8)
    assert rows.shape == (iters, 6) and n_iter == iters
    assert np.array_equal(rows, log[:, :6])
    assert np.all(rows[:, 2] == n)
    m, s, c = oracle.combine(list(log[:, 4]), list(log[:, 5]))
    assert abs(mean - m) <= 1e-12 * abs(m) and abs(sigma - s) <= 1e-12 * s
