"""Sharding one integral over ranks (CPU: the oracle computes each rank's
share; process groups use gloo)."""
import os
import socket

import numpy as np
import pytest
import torch

import oracle
from paper_2002_12921_b300 import workloads as W
from paper_2002_12921_b300.shard import (GridMismatch, RankFailure, ShardedVegas, VirtualRanks,
                                         grid_digest_host, shard_range)
from tests.shard_workers import OracleEngine, PerturbingEngine, gloo_worker

P = W.gauss_params(3, 0.15, [0.4, 0.5, 0.6])
SCHED = [(30_000, 1), (30_000, 1), (20_000, 1), (40_001, 0)]


# fixed-grid runs of two lengths, an adapting iteration between them
SCHED_F = [(30_000, 1), (20_000, 0), (20_000, 0), (25_000, 1), (40_001, 0), (40_001, 0),
           (30_000, 0)]


def single(sched=SCHED):
    return oracle.run(3, 20, 4, W.GAUSS, P, sched)


def assert_same_as_single(rows, grid, ref, sched=SCHED):
    assert len(rows) == len(sched)
    for t, r in enumerate(ref["log"]):
        assert rows[t][2] == sched[t][0]
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


def _spawn(tmp_path, fail_rank=-1, fail_iter=-1, perturb_rank=-1, defer=False,
           defer_fixed=False, sched=SCHED):
    spec = {"engine": (3, 20, 4, W.GAUSS, P), "schedule": sched, "alpha": 1.5}
    ctx = torch.multiprocessing.get_context("spawn")
    port = _port()
    procs = [ctx.Process(target=gloo_worker, args=(r, 2, port, str(tmp_path), spec, fail_rank,
                                                   fail_iter, perturb_rank, defer, defer_fixed))
             for r in range(2)]
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


def test_gloo_grids_that_differ_by_one_ulp_are_detected(tmp_path):
    """Rank 1's grid moves by one ulp in one edge after the second refinement
    (as if its totals had differed): the digest check after that refinement
    raises GridMismatch on both ranks, before either runs another iteration."""
    codes = _spawn(tmp_path, perturb_rank=1)
    assert codes == [0, 0]
    for r in range(2):
        err = (tmp_path / f"error{r}.txt").read_text()
        assert "GridMismatch" in err and "after 2 refinements" in err, err
        assert not os.path.exists(tmp_path / f"rows{r}.npy")


def test_gloo_deferred_checks_report_the_first_divergence(tmp_path):
    """The same one-ulp divergence with the checks deferred: the ranks finish
    the schedule without a host read of any digest, and verify() raises
    GridMismatch on both ranks naming the first check that differed (after
    the second refinement); without a divergence the deferred run equals the
    single run."""
    codes = _spawn(tmp_path, perturb_rank=1, defer=True)
    assert codes == [0, 0]
    for r in range(2):
        err = (tmp_path / f"error{r}.txt").read_text()
        assert "GridMismatch" in err and "after 2 refinements" in err, err
        assert "verify" in err
    ok = tmp_path / "ok"
    ok.mkdir()
    assert _spawn(ok, defer=True) == [0, 0]
    ref = single()
    for r in range(2):
        assert_same_as_single(np.load(ok / f"rows{r}.npy"), np.load(ok / f"grid{r}.npy"), ref)


def test_gloo_deferred_fixed_rows_equal_single_run(tmp_path):
    """Fixed-grid iterations exchanged in groups (ShardedVegas defer_fixed:
    each group of consecutive fixed-grid iterations of one n in one
    all-reduce, flushed before the next adapting iteration, on a change of n
    and at the end): the two ranks' logs and grids equal the single run's, in
    both layouts of the schedule, as with one exchange per iteration."""
    for sched in (SCHED_F, SCHED):
        out = tmp_path / f"s{len(sched)}"
        out.mkdir()
        assert _spawn(out, defer_fixed=True, sched=sched) == [0, 0]
        ref = single(sched)
        for r in range(2):
            assert_same_as_single(np.load(out / f"rows{r}.npy"), np.load(out / f"grid{r}.npy"),
                                  ref, sched)


def test_deferred_fixed_rows_single_process():
    """World size 1 (no process group): the deferred rows hold the rank's own
    sums until flush(), which installs the same totals a per-iteration
    exchange gives."""
    a, b = OracleEngine(3, 20, 4, W.GAUSS, P), OracleEngine(3, 20, 4, W.GAUSS, P)
    sa, sb = ShardedVegas(a, defer_fixed=True), ShardedVegas(b)
    for n, adapt in SCHED_F[:3]:
        sa.iterate(n, adapt)
        sb.iterate(n, adapt)
    assert sa.fixed == [1, 2, 20_000] and np.isnan(a.rows()[1, 4])
    sa.flush()
    assert sa.fixed is None
    assert np.array_equal(a.rows(), b.rows())


def test_virtual_ranks_detect_a_diverged_grid():
    engines = [OracleEngine(3, 20, 4, W.GAUSS, P), PerturbingEngine(3, 20, 4, W.GAUSS, P, at=0)]
    with pytest.raises(GridMismatch):
        VirtualRanks(engines).run(SCHED)


def _digest_by_definition(edges):
    """sum_i bits(e_i) (splitmix64(i) | 1) mod 2^64 with Python integers, where
    splitmix64(i) is output i of Vigna's SplitMix64 generator run as published:
    a 64-bit state starting at 0, advanced by the golden-ratio increment
    before each output is mixed."""
    m = (1 << 64) - 1
    bits = np.ascontiguousarray(edges, dtype=np.float64).ravel().view(np.uint64)
    state, total = 0, 0
    for b in bits:
        state = (state + 0x9E3779B97F4A7C15) & m
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        z ^= z >> 31
        total = (total + int(b) * (z | 1)) & m
    return total


def test_grid_digest_definition_and_sensitivity():
    """The host digest equals its definition computed with Python integers
    and the generator run step by step; equal grids give equal digests; moving
    any single edge by one ulp changes the digest."""
    e = oracle.refine(oracle.uniform_grid(3, 20), np.arange(60.0).reshape(3, 20) + 1.0, 1.5)
    d = grid_digest_host(e)
    h = _digest_by_definition(e)
    assert int(d[0]) & ((1 << 64) - 1) == h
    assert int(d[1]) == ~int(d[0])
    assert np.array_equal(grid_digest_host(e.copy()), d)
    for k in range(3):
        for j in range(21):
            f = e.copy()
            f[k, j] = np.nextafter(f[k, j], 2.0)
            assert grid_digest_host(f)[0] != d[0], (k, j)
