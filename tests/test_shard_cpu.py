"""Sharding one integral over ranks (CPU: the oracle computes each rank's
share; process groups use gloo)."""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_2002_12921_b300 import workloads as W
from paper_2002_12921_b300.shard import RankFailure, VirtualRanks, shard_range
from tests.shard_workers import OracleEngine, gloo_worker

P = W.gauss_params(3, 0.15, [0.4, 0.5, 0.6])
SCHED = [(30_000, 1), (30_000, 1), (20_000, 1), (40_001, 0)]


def single():
    return oracle.run(3, 20, 4, W.GAUSS, P, SCHED)


def assert_same_as_single(rows, grid, ref):
    for t, r in enumerate(ref["log"]):
        assert rows[t][2] == SCHED[t][0]
        assert abs(rows[t][4] - r["I"]) <= 1e-12 * abs(r["I"]), t
        assert abs(rows[t][5] - r["var"]) <= 1e-10 * r["var"], t
    assert np.allclose(grid, ref["edges"], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n,world", [(10, 3), (1000, 7), (2**40 + 3, 8), (5, 5)])
def test_shard_ranges_partition_the_indices(n, world):
    r = [shard_range(n, k, world) for k in range(world)]
    assert r[0][0] == 0 and r[-1][1] == n
    assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
    assert all(e - b in (n // world, n // world + 1) for b, e in r)


@pytest.mark.parametrize("world", [1, 2, 3])
def test_virtual_ranks_equal_single_run(world):
    engines = [OracleEngine(3, 20, 4, W.GAUSS, P) for _ in range(world)]
    VirtualRanks(engines).run(SCHED)
    ref = single()
    for eng in engines:
        assert_same_as_single(eng.rows(), eng.grid(), ref)


def test_virtual_rank_failure_is_retried_exactly():
    def fault(rank, iteration, attempt):
        if (rank, iteration, attempt) in {(1, 2, 0), (0, 3, 0), (0, 3, 1)}:
            raise RankFailure("injected")

    engines = [OracleEngine(3, 20, 4, W.GAUSS, P) for _ in range(2)]
    vr = VirtualRanks(engines, fault=fault)
    vr.run(SCHED)
    assert [(f[0], f[1], f[2]) for f in vr.failures] == [(2, 1, 0), (3, 0, 0), (3, 0, 1)]
    assert_same_as_single(engines[0].rows(), engines[0].grid(), single())


def test_virtual_rank_that_keeps_failing_is_reported():
    def fault(rank, iteration, attempt):
        if rank == 1 and iteration == 1:
            raise RankFailure("down")

    vr = VirtualRanks([OracleEngine(3, 20, 4, W.GAUSS, P) for _ in range(2)], fault=fault)
    with pytest.raises(RankFailure):
        vr.run(SCHED)


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(tmp_path, fail_rank=-1, fail_iter=-1):
    spec = {"engine": (3, 20, 4, W.GAUSS, P), "schedule": SCHED, "alpha": 1.5}
    ctx = torch.multiprocessing.get_context("spawn")
    port = _port()
    procs = [ctx.Process(target=gloo_worker, args=(r, 2, port, str(tmp_path), spec, fail_rank,
                                                   fail_iter)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    return codes


def test_gloo_two_ranks_equal_single_run(tmp_path):
    codes = _spawn(tmp_path)
    assert codes == [0, 0]
    ref = single()
    for r in range(2):
        assert_same_as_single(np.load(tmp_path / f"rows{r}.npy"),
                              np.load(tmp_path / f"grid{r}.npy"), ref)


def test_gloo_rank_failure_is_detected_by_its_peer(tmp_path):
    """Rank 1 dies (host side) before its share of iteration 2; rank 0's next
    all-reduce ends with an error instead of waiting forever."""
    codes = _spawn(tmp_path, fail_rank=1, fail_iter=2)
    assert codes[1] == 3
    assert os.path.exists(tmp_path / "error0.txt")
    assert not os.path.exists(tmp_path / "rows0.npy")
