"""CPU engines and process-group workers for the sharding tests (test
infrastructure: the oracle computes each rank's share)."""
import os
import sys
import traceback
from datetime import timedelta

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_12921_b300.shard import ShardedVegas, grid_digest_host  # noqa: E402


class OracleEngine:
    """One rank's engine computed by the FP64 oracle."""

    def __init__(self, dim, nbins, seed, fid, params):
        self.dim, self.nbins, self.seed, self.fid, self.params = dim, nbins, seed, fid, params
        self.e = oracle.uniform_grid(dim, nbins)
        self.it = 0
        self.part = None
        self.hist = np.zeros((dim, nbins))
        self._rows = []

    def iterate_range(self, n, begin, end, adapt):
        """This rank's share of iteration self.it; its row holds the share's
        sums until an import replaces them (as a device state's log does)."""
        self.part = oracle.iterate_range(self.e, self.seed, self.it, begin, end - begin, self.fid,
                                         self.params, adapt)
        if self.part["hist"] is None:
            self.part["hist"] = np.zeros((self.dim, self.nbins))
        p = self.part
        self._rows.append([p["S1"], p["S2"], end - begin, float(p["nonfinite"]), np.nan, np.nan])
        self.it += 1
        return len(self._rows) - 1

    def export(self):
        p = self.part
        return torch.tensor([p["S1"], p["S2"], float(p["nonfinite"])] + list(p["hist"].ravel()),
                            dtype=torch.float64)

    def _install(self, row, s1, s2, nonfinite, n):
        I, var = oracle.estimate(float(s1), float(s2), n)
        self._rows[row] = [s1, s2, n, nonfinite, I, var]

    def import_(self, totals, n):
        t = totals.numpy()
        self._install(len(self._rows) - 1, t[0], t[1], t[2], n)
        self.hist = t[3:].reshape(self.dim, self.nbins).copy()

    def export_rows(self, first, count):
        rows = self._rows[first:first + count]
        return torch.tensor([v for r in rows for v in (r[0], r[1], r[3])], dtype=torch.float64)

    def import_rows(self, first, count, totals, n):
        t = totals.numpy().reshape(count, 3)
        for r in range(count):
            self._install(first + r, t[r, 0], t[r, 1], t[r, 2], n)

    def refine(self, alpha):
        self.e = oracle.refine(self.e, self.hist, alpha)

    def rows(self):
        return np.array(self._rows)

    def grid(self):
        return self.e

    def grid_digest(self):
        return torch.from_numpy(grid_digest_host(self.e))


class PerturbingEngine(OracleEngine):
    """An oracle engine whose refinement after iteration `at` moves one
    interior edge by one ulp (a rank that received different totals)."""

    def __init__(self, *args, at=1, edge=(0, 3)):
        super().__init__(*args)
        self.at, self.edge = at, edge

    def refine(self, alpha):
        super().refine(alpha)
        if self.it - 1 == self.at:
            self.e = self.e.copy()
            self.e[self.edge] = np.nextafter(self.e[self.edge], 2.0)


def gloo_worker(rank, world, port, out_dir, spec, fail_rank, fail_iter, perturb_rank=-1,
                defer=False, defer_fixed=False):
    """One gloo rank: run the sharded schedule and save rows and grid; the rank
    `fail_rank` raises (host side) before its share of iteration `fail_iter`;
    the others record the error their next collective reports.  The rank
    `perturb_rank` moves one edge of its grid by one ulp after the refinement
    of iteration 1 (every rank must then raise GridMismatch).  defer: the
    digest checks are deferred and verified once, after the schedule.
    defer_fixed: fixed-grid rows are exchanged together (ShardedVegas.flush)."""
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=timedelta(seconds=20))
    eng = (PerturbingEngine(*spec["engine"], at=1) if rank == perturb_rank
           else OracleEngine(*spec["engine"]))
    sv = ShardedVegas(eng, defer_checks=defer, defer_fixed=defer_fixed)
    try:
        for t, (n, adapt) in enumerate(spec["schedule"]):
            if rank == fail_rank and t == fail_iter:
                raise RuntimeError("injected failure")
            sv.iterate(n, adapt, spec["alpha"])
        sv.flush()
        sv.check_grids()
        sv.verify()
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), eng.rows())
        np.save(os.path.join(out_dir, f"grid{rank}.npy"), eng.grid())
    except Exception:
        with open(os.path.join(out_dir, f"error{rank}.txt"), "w") as fh:
            fh.write(traceback.format_exc())
        if rank == fail_rank:
            os._exit(3)  # the failing rank leaves without further collectives
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass
