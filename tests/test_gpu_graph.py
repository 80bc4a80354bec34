"""A state's schedule captured into a CUDA graph (Vegas.capture): replays run
further iterations with fresh counters, exactly as the same schedule enqueued
again would (the iteration number and the log row come from device memory),
and a replay past the log's capacity does nothing and is reported."""
import numpy as np
import pytest

import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SCHED = [(300_000, 1)] * 3 + [(700_001, 0)] * 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
@pytest.mark.parametrize("chunk", [0, 250_000])
def test_replays_equal_the_schedule_enqueued_again(mode, chunk):
    p = W.gauss_params(6, 0.12, np.linspace(0.35, 0.65, 6))
    stream = torch.cuda.Stream()
    eager = V.Vegas(6, 40, 9, mode, W.GAUSS, p, max_iters=16, stream=stream)
    graphed = V.Vegas(6, 40, 9, mode, W.GAUSS, p, max_iters=16, stream=stream)
    for v in (eager, graphed):
        v.config(chunk_samples=chunk)
    for _ in range(3):
        eager.run(SCHED)
    g = graphed.capture(SCHED)
    assert graphed.iterations().shape[0] == 0  # the capture ran nothing
    for _ in range(3):
        g.replay()
    re, rg = eager.iterations(), graphed.iterations()
    assert re.shape == rg.shape == (15, 6)
    tol = 1e-13 if mode == V.VEGAS_FP64 else 1e-5
    assert np.array_equal(re[:, 2:4], rg[:, 2:4])
    assert np.allclose(rg[:, 4], re[:, 4], rtol=tol, atol=0)
    assert np.allclose(graphed.grid(), eager.grid(), rtol=0, atol=10 * tol)
    me, mg = eager.result(3)[0], graphed.result(3)[0]
    assert abs(me - mg) <= 10 * tol * abs(me)
    eager.close()
    graphed.close()


def test_a_replay_past_the_log_capacity_is_reported():
    p = W.gauss_params(3, 0.2)
    with pytest.raises(ValueError):  # CUDA does not capture the default stream
        V.Vegas(3, 20, 1, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=5,
                stream=torch.cuda.default_stream()).capture(SCHED)
    v = V.Vegas(3, 20, 1, V.VEGAS_FP32_EVAL, W.GAUSS, p, max_iters=5, stream=torch.cuda.Stream())
    g = v.capture(SCHED)  # five iterations: the whole log
    g.replay()
    assert v.result(0)[3] == 5
    grid = v.grid()
    g.replay()  # nothing left: every iteration of this replay returns at once
    with pytest.raises(V.VegasError) as e:
        v.result(0)
    assert e.value.status == V.VEGAS_ESTATE
    assert np.array_equal(v.grid(), grid)  # refinements of an empty histogram keep the grid
    v.close()
