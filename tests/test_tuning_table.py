"""The autotuner's JSON table (binding.TuningTable), host logic only: a shape
is tuned once, stored under its key, read back by a new table object from the
file, and distinct shapes / sample-count decades get distinct entries."""
import json

from paper_2002_12921_b300 import binding as B


def test_tuning_table_tunes_once_and_persists(tmp_path):
    calls = []

    def fake_tuner(dim, nbins, mode, integrand, params, n, adapt=False):
        calls.append((dim, nbins, mode, integrand, n, adapt))
        return dict(block_threads=128 if dim > 4 else 256, blocks_per_sm=0,
                    min_samples_per_thread=8), {}

    path = str(tmp_path / "tuning.json")
    t = B.TuningTable(path, tuner=fake_tuner)
    a = t.lookup(8, 50, B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, [0.1] + [0.5] * 8, 10_000_000, True)
    b = t.lookup(8, 50, B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, [0.1] + [0.5] * 8, 30_000_000, True)
    assert a == b == dict(block_threads=128, blocks_per_sm=0, min_samples_per_thread=8)
    assert len(calls) == 1  # same decade of n: one tuning
    t.lookup(8, 50, B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, [0.1] + [0.5] * 8, 100_000_000, False)
    t.lookup(3, 50, B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, [0.1] + [0.5] * 3, 100_000_000, False)
    assert len(calls) == 3
    stored = json.load(open(path))
    assert len(stored) == 3
    assert B.TuningTable.key(B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, 8, 50, 10_000_000, True) in stored
    fresh = B.TuningTable(path, tuner=fake_tuner)  # a later process
    assert fresh.lookup(3, 50, B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS, [0.1] + [0.5] * 3,
                        500_000_000, False)["block_threads"] == 256
    assert len(calls) == 3


class FakeBatch:
    """The attributes and configuration calls TuningTable.lookup_batch uses."""

    def __init__(self, dims, n):
        self.dims, self.n_samples, self.nbins = dims, n, 50
        self.mode, self.integrand = B.VEGAS_FP32_EVAL, B.VEGAS_GAUSS
        self.calls = []

    def config(self, block_threads=0, tile_samples=0):
        self.calls.append(("config", block_threads, tile_samples))

    def config_tiles_by_dim(self, tiles):
        self.calls.append(("tiles", dict(tiles)))

    def reset(self):
        self.calls.append(("reset",))


def test_batch_entries_are_kept_per_dimension_bucket(tmp_path):
    """A batch is tuned once; its entry holds the block size, the batch-wide
    tile and one tile per dimension bucket, and configures a later batch of
    the same key (in another process) without tuning: every dimension of a
    bucket gets the bucket's tile."""
    tuned = []

    def fake_tuner(batch):
        tuned.append(batch)
        return (512, 8192, {2: 4096, 3: 4096, 9: 16384}), {}

    path = str(tmp_path / "tuning.json")
    t = B.TuningTable(path)
    a = FakeBatch([2, 3, 9], [10_000, 20_000, 30_000])
    e = t.lookup_batch(a, tuner=fake_tuner)
    assert e == {"block_threads": 512, "tile_samples": 8192,
                 "tiles_by_bucket": {"1-4": 4096, "9-12": 16384}}
    assert ("config", 512, 8192) in a.calls and a.calls[-1] == ("reset",)
    b = FakeBatch([2, 3, 9], [15_000, 20_000, 40_000])  # same buckets, count and decade
    fresh = B.TuningTable(path)
    assert fresh.lookup_batch(b, tuner=fake_tuner) == e
    assert len(tuned) == 1
    assert ("tiles", {2: 4096, 3: 4096, 9: 16384}) in b.calls
    c = FakeBatch([2, 3, 17], [10_000, 20_000, 30_000])  # another bucket: tuned anew
    fresh.lookup_batch(c, tuner=fake_tuner)
    assert len(tuned) == 2 and B.TuningTable.batch_key(c) != B.TuningTable.batch_key(a)
