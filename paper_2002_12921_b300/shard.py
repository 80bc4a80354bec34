"""One Vegas integral sharded over several devices.

Sample indices are global and every sample is a pure function of its
counter, so one iteration of n samples splits into contiguous index ranges
that different devices (ranks) compute independently.  The only exchange is
one sum per iteration of {S1, S2, nonfinite, histogram} (3 + d N doubles);
after it every rank holds the totals and refines identically, so the grids
never diverge and the result equals a single device's run up to the order of
the sums.  (VegasFlow Sec. 3.4 distributes events over devices of one
machine; this is that split, written for counter-based sampling.)  Fixed-grid
iterations need no exchange before the combination, so a run of them can
share one sum of 3 doubles per row (``defer_fixed``).

Identical grids rest on every rank receiving bit-identical totals from the
all-reduce.  ``ShardedVegas`` checks that they did: after every
``check_every``-th refinement (and on request) each rank reduces a 64-bit digest
of its grid's bit patterns with MAX, paired with its complement (so one
16-byte all-reduce gives the largest and the smallest digest), and every rank
raises ``GridMismatch`` when they differ.  Cost per check: one digest kernel,
one 16-byte all-reduce and one host read of its result (a stream
synchronisation), or, with ``defer_checks``, no host read until ``verify()``.

An engine is what one rank computes with; it provides
    iterate_range(n, begin, end, adapt) -> the iteration's log row,
    export() -> 1-d tensor,
    import_(totals, n), refine(alpha), rows(), grid(),
    grid_digest() -> int64 tensor [digest, ~digest] on the collective's device,
and, for deferred fixed-grid exchanges, export_rows(first, count) -> 1-d tensor
of {S1, S2, nonfinite} per row and import_rows(first, count, totals, n).
``GpuShardEngine`` wraps a CUDA ``Vegas`` state (vegas_iterate_range /
vegas_shard_export / vegas_shard_import / vegas_grid_digest); tests plug in
CPU engines.
"""
import logging

import numpy as np

log = logging.getLogger(__name__)

_M64 = (1 << 64) - 1


def _splitmix64(i):
    """Vigna's SplitMix64 output function of the uint64 array i."""
    with np.errstate(over="ignore"):
        z = (i + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def grid_digest_host(edges):
    """The digest vegas_grid_digest defines, of a host grid (dim x (nbins+1)
    doubles, row-major): sum_i bits(e_i) (splitmix64(i) | 1) mod 2^64, as a
    signed 64-bit pair [digest, ~digest]."""
    bits = np.ascontiguousarray(edges, dtype=np.float64).ravel().view(np.uint64)
    k = _splitmix64(np.arange(bits.size, dtype=np.uint64)) | np.uint64(1)
    with np.errstate(over="ignore"):
        h = int(np.sum(bits * k, dtype=np.uint64))
    return np.array([h, ~h & _M64], dtype=np.uint64).view(np.int64)


def shard_range(n, rank, world):
    """Contiguous share [begin, end) of n sample indices for `rank` of `world`."""
    return n * rank // world, n * (rank + 1) // world


class GpuShardEngine:
    """A rank's engine over a CUDA ``Vegas`` state."""

    def __init__(self, vegas, logged=None):
        """logged: the log rows the state already holds (0 for a new state);
        None reads them from the state (one stream synchronisation)."""
        import torch

        from . import binding as B

        self.v, self.B = vegas, B
        self.buf = torch.zeros(3 + vegas.dim * vegas.nbins, dtype=torch.float64,
                               device=vegas.workspace.device)
        self.digest = torch.zeros(2, dtype=torch.int64, device=vegas.workspace.device)
        # log rows the state already holds (a resumed state continues after them)
        self.logged = len(vegas.iterations()) if logged is None else int(logged)

    def iterate_range(self, n, begin, end, adapt):
        """Enqueue this rank's range; returns the iteration's log row."""
        rc = self.B.lib().vegas_iterate_range(self.v.handle, int(n), int(begin), int(end),
                                              1 if adapt else 0)
        if rc == self.B.VEGAS_ECUDA:
            # a launch of this rank's range failed.  Run again, the range
            # reproduces its samples exactly when the failure came before the
            # first launch (an injected failure, a launch-configuration error);
            # the iteration's log row and count are written only on success
            raise RankFailure("vegas_iterate_range: " + self.B.lib().vegas_strerror(rc).decode())
        self.B._check(rc, "vegas_iterate_range")
        self.logged += 1
        return self.logged - 1

    def export(self):
        self.B._check(self.B.lib().vegas_shard_export(self.v.handle, self.buf.data_ptr()),
                      "vegas_shard_export")
        return self.buf

    def import_(self, totals, n):
        # the library reads exactly 3 + dim * nbins doubles of device memory
        if (totals.numel() != self.buf.numel() or totals.dtype != self.buf.dtype
                or totals.device != self.buf.device or not totals.is_contiguous()):
            raise ValueError(f"totals must be a contiguous float64 tensor of "
                             f"{self.buf.numel()} elements on {self.buf.device}")
        self.B._check(self.B.lib().vegas_shard_import(self.v.handle, totals.data_ptr(), int(n)),
                      "vegas_shard_import")

    def export_rows(self, first, count):
        import torch

        buf = torch.empty(3 * count, dtype=torch.float64, device=self.buf.device)
        self.B._check(self.B.lib().vegas_shard_export_rows(self.v.handle, int(first), int(count),
                                                            buf.data_ptr()),
                      "vegas_shard_export_rows")
        return buf

    def import_rows(self, first, count, totals, n):
        # the library reads exactly 3 * count doubles of device memory
        if (totals.numel() != 3 * count or totals.dtype != self.buf.dtype
                or totals.device != self.buf.device or not totals.is_contiguous()):
            raise ValueError(f"totals must be a contiguous float64 tensor of {3 * count} "
                             f"elements on {self.buf.device}")
        self.B._check(self.B.lib().vegas_shard_import_rows(self.v.handle, int(first), int(count),
                                                            totals.data_ptr(), int(n)),
                      "vegas_shard_import_rows")

    def refine(self, alpha):
        self.v.refine(alpha)

    def rows(self):
        return self.v.iterations()

    def grid(self):
        return self.v.grid()

    def grid_digest(self):
        self.B._check(self.B.lib().vegas_grid_digest(self.v.handle, self.digest.data_ptr()),
                      "vegas_grid_digest")
        return self.digest


class RankFailure(RuntimeError):
    """Raised (host side) by a rank that could not produce its share."""


class GridMismatch(RankFailure):
    """Raised on every rank when the ranks' grids differ after a refinement."""


class ShardedVegas:
    """Drives one engine per rank of a torch.distributed process group: each
    iteration computes this rank's index range, all-reduces the partial sums
    (NCCL for CUDA tensors, gloo for CPU ones) and refines.  Every iteration
    needs n >= world size.  check_every = k > 0: after every k-th adapting
    iteration the ranks compare grid digests (check_grids); 0: only when
    check_grids() is called (run() calls it at the end).

    defer_checks=True: a check all-reduces the digests as usual but leaves the
    result on the device, so no check synchronises the host with the stream in
    the middle of a schedule; verify() (called by run() at the end) reads every
    pending result and raises GridMismatch for the first that differs.

    defer_fixed=True: consecutive fixed-grid iterations of the same n keep their
    rank-local sums until flush() (called before the next adapting iteration,
    by run() at the end, and by the caller before reading the log) sums all of
    their rows in one all-reduce of 3 doubles per row: a fixed-grid iteration
    changes neither grid nor histogram, so nothing before the combination
    needs its totals."""

    def __init__(self, engine, group=None, check_every=1, defer_checks=False,
                 defer_fixed=False):
        import torch.distributed as dist

        self.engine, self.group, self.dist = engine, group, dist
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1
        self.check_every = check_every
        self.defer_checks = defer_checks
        self.defer_fixed = defer_fixed
        self.pending = []  # (refinements, reduced digest pair) awaiting verify()
        self.fixed = None  # [first row, count, n] of fixed-grid rows awaiting flush()
        self.refinements = 0

    def iterate(self, n, adapt, alpha=1.5):
        if n < self.world:
            raise ValueError("need at least one sample per rank")
        begin, end = shard_range(n, self.rank, self.world)
        if adapt or not self.defer_fixed or (self.fixed is not None and self.fixed[2] != n):
            self.flush()
        t = self.engine.iterate_range(n, begin, end, adapt)  # the iteration's log row
        if not adapt and self.defer_fixed:
            if self.fixed is None:
                self.fixed = [t, 1, n]
            else:
                self.fixed[1] += 1
            return
        totals = self.engine.export()
        if self.world > 1:
            self.dist.all_reduce(totals, op=self.dist.ReduceOp.SUM, group=self.group)
        self.engine.import_(totals, n)
        if adapt:
            self.engine.refine(alpha)
            self.refinements += 1
            if self.check_every and self.refinements % self.check_every == 0:
                self.check_grids()

    def flush(self):
        """Exchange the deferred fixed-grid rows (one all-reduce), if any."""
        if self.fixed is None:
            return
        first, count, n = self.fixed
        self.fixed = None
        totals = self.engine.export_rows(first, count)
        if self.world > 1:
            self.dist.all_reduce(totals, op=self.dist.ReduceOp.SUM, group=self.group)
        self.engine.import_rows(first, count, totals, n)

    def check_grids(self):
        """Raise GridMismatch (on every rank) unless all ranks' grids have the
        same digest: one all-reduce of [digest, ~digest] with MAX gives the
        largest digest and the complement of the smallest.  With defer_checks
        the reduced pair is kept for verify() instead of read here."""
        d = self.engine.grid_digest().clone()
        if self.world > 1:
            self.dist.all_reduce(d, op=self.dist.ReduceOp.MAX, group=self.group)
        if self.defer_checks:
            self.pending.append((self.refinements, d))
            return
        self._raise_if_differ(self.refinements, d)

    def verify(self):
        """Read the deferred checks' results (one host synchronisation) and
        raise GridMismatch for the first whose digests differ."""
        pending, self.pending = self.pending, []
        for refinements, d in pending:
            self._raise_if_differ(refinements, d)

    def _raise_if_differ(self, refinements, d):
        hi, lo = int(d[0]), ~int(d[1])
        if hi != lo:
            raise GridMismatch(f"rank {self.rank}: grids differ across ranks after "
                               f"{refinements} refinements (digests {lo:#x} .. {hi:#x})")

    def run(self, schedule, alpha=1.5):
        for n, adapt in schedule:
            self.iterate(n, adapt, alpha)
        self.flush()
        self.check_grids()
        self.verify()


class VirtualRanks:
    """`world` ranks emulated one after another in this process, each with its
    own engine (on one GPU, or on the CPU), summing their exported partials on
    the host side of the exchange.  A rank whose step raises RankFailure before
    contributing is re-run: its counter range is deterministic, so the retry
    reproduces exactly what the rank would have produced.  `fault` is an
    optional hook fault(rank, iteration, attempt) that may raise RankFailure."""

    def __init__(self, engines, fault=None, max_retries=2):
        self.engines, self.fault, self.max_retries = list(engines), fault, max_retries
        self.world = len(self.engines)
        self.iteration = 0
        self.failures = []

    def _contribute(self, r, n, adapt):
        begin, end = shard_range(n, r, self.world)
        for attempt in range(self.max_retries + 1):
            try:
                if self.fault is not None:
                    self.fault(r, self.iteration, attempt)
                self.engines[r].iterate_range(n, begin, end, adapt)
                return self.engines[r].export().clone()
            except RankFailure as exc:
                self.failures.append((self.iteration, r, attempt, str(exc)))
                log.warning("rank %d failed at iteration %d (attempt %d): %s; re-running "
                            "its range [%d, %d)", r, self.iteration, attempt, exc, begin, end)
        raise RankFailure(f"rank {r} failed {self.max_retries + 1} times at iteration "
                          f"{self.iteration}")

    def iterate(self, n, adapt, alpha=1.5):
        if n < self.world:
            raise ValueError("need at least one sample per rank")
        totals = None
        for r in range(self.world):
            part = self._contribute(r, n, adapt)
            totals = part if totals is None else totals + part
        for eng in self.engines:
            eng.import_(totals, n)
            if adapt:
                eng.refine(alpha)
        if adapt:
            digests = {tuple(int(x) for x in eng.grid_digest()) for eng in self.engines}
            if len(digests) != 1:
                raise GridMismatch(f"virtual ranks' grids differ after iteration "
                                   f"{self.iteration}")
        self.iteration += 1

    def run(self, schedule, alpha=1.5):
        for n, adapt in schedule:
            self.iterate(n, adapt, alpha)
