"""Virtual ranks on one GPU: each rank is its own Vegas state computing its
share of the counter range (vegas_iterate_range), the partial sums are added
(vegas_shard_export / vegas_shard_import) and every rank refines; the result
must equal one state's run and the FP64 oracle."""
import numpy as np
import pytest

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W
from paper_2002_12921_b300.shard import (GpuShardEngine, RankFailure, VirtualRanks,
                                         shard_range)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

P = W.gauss_params(6, 0.12, [0.3, 0.4, 0.5, 0.5, 0.6, 0.7])
SCHED = [(300_000, 1), (300_000, 1), (200_001, 1), (500_000, 0)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


def fp64_tol(edges):
    return max(1e-12, 8 * edges.shape[0] * np.finfo(float).eps / np.min(np.diff(edges, axis=1)))


@pytest.mark.parametrize("world", [2, 3])
def test_gpu_virtual_ranks_fp64_equal_oracle(world):
    states = [V.Vegas(6, 40, 21, V.VEGAS_FP64, W.GAUSS, P, max_iters=8) for _ in range(world)]
    VirtualRanks([GpuShardEngine(s) for s in states]).run(SCHED)
    ref = oracle.run(6, 40, 21, W.GAUSS, P, SCHED, nthreads=8)
    for s in states:
        rows = s.iterations()
        for t, r in enumerate(ref["log"]):
            tol = 1e-12 if t == 0 else fp64_tol(ref["grids"][t])
            assert rows[t][2] == SCHED[t][0]
            assert abs(rows[t][4] - r["I"]) <= tol * abs(r["I"]), t
        assert np.allclose(s.grid(), ref["edges"], rtol=1e-12, atol=1e-15)
        s.close()


def test_gpu_virtual_ranks_fp32_match_one_state_and_survive_a_failure():
    def fault(rank, iteration, attempt):
        if (rank, iteration, attempt) == (1, 1, 0):
            raise RankFailure("injected")

    one = V.Vegas(6, 40, 21, V.VEGAS_FP32_EVAL, W.GAUSS, P, max_iters=8)
    one.run(SCHED)
    ref = one.iterations()
    states = [V.Vegas(6, 40, 21, V.VEGAS_FP32_EVAL, W.GAUSS, P, max_iters=8) for _ in range(2)]
    vr = VirtualRanks([GpuShardEngine(s) for s in states], fault=fault)
    vr.run(SCHED)
    assert len(vr.failures) == 1
    for s in states:
        rows = s.iterations()
        # float histograms summed per shard round differently: the FP32 bound
        assert np.allclose(rows[:, 4], ref[:, 4], rtol=1e-5, atol=0)
        assert np.allclose(s.grid(), one.grid(), rtol=0, atol=1e-6)
        s.close()
    one.close()


def test_a_failed_launch_is_retried_and_the_run_stays_exact():
    """A rank whose range launch fails (vegas_inject_failure: VEGAS_ECUDA
    before anything is enqueued) is re-run by the coordinator; the result
    equals the oracle's, and a state's own next call after a failure works."""
    states = [V.Vegas(6, 40, 21, V.VEGAS_FP64, W.GAUSS, P, max_iters=8) for _ in range(2)]
    states[1].inject_failure(3)  # its third enqueueing call: iteration 1's range
    vr = VirtualRanks([GpuShardEngine(s) for s in states])
    vr.run(SCHED)
    assert [(f[0], f[1]) for f in vr.failures] == [(1, 1)]
    ref = oracle.run(6, 40, 21, W.GAUSS, P, SCHED, nthreads=8)
    for s in states:
        rows = s.iterations()
        for t, r in enumerate(ref["log"]):
            tol = 1e-12 if t == 0 else fp64_tol(ref["grids"][t])
            assert abs(rows[t][4] - r["I"]) <= tol * abs(r["I"]), t
        s.close()
    v = V.Vegas(3, 10, 1, V.VEGAS_FP32_EVAL, W.GAUSS, W.gauss_params(3, 0.2), max_iters=4)
    v.inject_failure(1)
    with pytest.raises(V.VegasError) as e:
        v.iterate(10_000, 1)
    assert e.value.status == V.VEGAS_ECUDA
    v.inject_failure(1)
    with pytest.raises(V.VegasError):
        v.refine()
    v.run([(10_000, 1), (10_000, 0)])  # the state is untouched and usable
    assert v.result(0)[3] == 2
    v.close()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_grid_digest_on_the_device_equals_its_host_definition(mode):
    """vegas_grid_digest (a kernel over the grid in device memory) equals the
    host digest of the same grid read back, on a uniform and on a refined
    grid; the pair's second word is the complement of the first; the virtual
    ranks' digests agree after every refinement."""
    from paper_2002_12921_b300.shard import grid_digest_host

    v = V.Vegas(6, 40, 21, mode, W.GAUSS, P, max_iters=4)
    eng = GpuShardEngine(v)
    for _ in range(2):
        d = eng.grid_digest().cpu().numpy().copy()
        assert np.array_equal(d, grid_digest_host(v.grid()))
        assert int(d[1]) == ~int(d[0])
        v.iterate(200_000, 1)
        v.refine(1.5)
    v.close()
    states = [V.Vegas(6, 40, 21, mode, W.GAUSS, P, max_iters=8) for _ in range(2)]
    VirtualRanks([GpuShardEngine(s) for s in states]).run(SCHED)  # digests checked inside
    for s in states:
        s.close()


def test_host_buffers_are_refused_where_device_memory_is_required():
    """A host buffer handed to the calls whose kernels write or read the
    caller's memory is refused with VEGAS_EINVAL before anything is enqueued."""
    import ctypes

    v = V.Vegas(3, 10, 1, V.VEGAS_FP64, W.GAUSS, W.gauss_params(3, 0.1), max_iters=2)
    v.iterate(10_000, 1)
    host = np.zeros(64)
    hp = ctypes.c_void_p(host.ctypes.data)
    L = V.lib()
    assert L.vegas_shard_export(v.handle, hp) == V.VEGAS_EINVAL
    assert L.vegas_shard_import(v.handle, hp, 10_000) == V.VEGAS_EINVAL
    assert L.vegas_shard_export_rows(v.handle, 0, 1, hp) == V.VEGAS_EINVAL
    assert L.vegas_shard_import_rows(v.handle, 0, 1, hp, 10_000) == V.VEGAS_EINVAL
    assert L.vegas_grid_digest(v.handle, hp) == V.VEGAS_EINVAL
    p = (ctypes.c_double * 4)(*W.gauss_params(3, 0.1))
    assert L.vegas_gauss_adjoint(v.handle, p, 4, 0, 10_000, 1, hp) == V.VEGAS_EINVAL
    assert L.vegas_sample_words(1, 0, 0, 0, 8, 3, hp,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) \
        == V.VEGAS_EINVAL
    torch.cuda.synchronize()
    assert np.all(host == 0.0)
    assert v.iterations().shape[0] == 1
    v.close()


def test_gpu_fixed_rows_exchanged_together_equal_oracle():
    """Two virtual ranks exchange an adapting iteration at once and then three
    fixed-grid iterations in one sum of their rows (vegas_shard_export_rows /
    vegas_shard_import_rows): every row equals the FP64 oracle's run, as with
    one exchange per iteration; rows outside the log are refused."""
    import ctypes

    sched = [(300_000, 1), (200_001, 0), (200_001, 0), (200_001, 0)]
    states = [V.Vegas(6, 40, 21, V.VEGAS_FP64, W.GAUSS, P, max_iters=8) for _ in range(2)]
    engs = [GpuShardEngine(s) for s in states]
    n = sched[0][0]
    for r, e in enumerate(engs):
        e.iterate_range(n, *shard_range(n, r, 2), True)
    tot = engs[0].export().clone() + engs[1].export().clone()
    for e in engs:
        e.import_(tot, n)
        e.refine(1.5)
    n = sched[1][0]
    for _ in range(3):
        for r, e in enumerate(engs):
            e.iterate_range(n, *shard_range(n, r, 2), False)
    rows = engs[0].export_rows(1, 3).clone() + engs[1].export_rows(1, 3).clone()
    for e in engs:
        e.import_rows(1, 3, rows, n)
    ref = oracle.run(6, 40, 21, W.GAUSS, P, sched, nthreads=8)
    buf = torch.zeros(12, dtype=torch.float64, device="cuda")
    L = V.lib()
    assert L.vegas_shard_export_rows(states[0].handle, 2, 3, ctypes.c_void_p(buf.data_ptr())) \
        == V.VEGAS_ESTATE
    assert L.vegas_shard_import_rows(states[0].handle, -1, 1, ctypes.c_void_p(buf.data_ptr()),
                                     n) == V.VEGAS_EINVAL
    for s in states:
        got = s.iterations()
        assert got.shape[0] == 4
        for t, r in enumerate(ref["log"]):
            tol = 1e-12 if t == 0 else fp64_tol(ref["grids"][t])
            assert got[t][2] == sched[t][0]
            assert abs(got[t][4] - r["I"]) <= tol * abs(r["I"]), t
            assert abs(got[t][5] - r["var"]) <= 1e3 * tol * r["var"], t
        assert np.allclose(s.grid(), ref["edges"], rtol=1e-12, atol=1e-15)
        s.close()


def test_deferred_fixed_rows_after_earlier_iterations():
    """A state that already logged iterations before ShardedVegas took it over
    (the engine reads how many): with defer_fixed, the next fixed-grid rows
    are exchanged into their own rows, and the log equals the same schedule
    run on one state call by call."""
    from paper_2002_12921_b300.shard import ShardedVegas

    sched = [(200_000, 1), (200_000, 1), (150_001, 0), (150_001, 0), (150_001, 0)]
    a = V.Vegas(6, 40, 9, V.VEGAS_FP64, W.GAUSS, P, max_iters=8)
    b = V.Vegas(6, 40, 9, V.VEGAS_FP64, W.GAUSS, P, max_iters=8)
    for n, adapt in sched[:2]:
        a.iterate(n, 1)
        a.refine(1.5)
    sv = ShardedVegas(GpuShardEngine(a), defer_fixed=True)
    assert sv.engine.logged == 2
    for n, adapt in sched[2:]:
        sv.iterate(n, adapt)
    assert sv.fixed == [2, 3, 150_001]
    sv.flush()
    b.run(sched)
    ra, rb = a.iterations(), b.iterations()
    assert ra.shape == rb.shape == (5, 6)
    assert np.array_equal(ra[:, 2:4], rb[:, 2:4])
    assert np.allclose(ra[:, [0, 1, 4, 5]], rb[:, [0, 1, 4, 5]], rtol=1e-13, atol=0)
    a.close()
    b.close()
