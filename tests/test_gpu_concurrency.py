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
