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
