"""Pins for the oracle's Philox4x32-10 and its counter layout (CPU only)."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _edge_counters(rng, n):
    """Random counters plus words at the carry boundaries 0, 1, 2^31, 2^32-1."""
    special = np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, 0xFFFFFFFF], dtype=np.uint32)
    c = rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    grid = np.array(np.meshgrid(special, special, special[:3], special[:3])).reshape(4, -1).T
    return np.concatenate([c, grid.astype(np.uint32)])


@pytest.mark.parametrize("seed", [0, 1, 2, 0xDEADBEEFCAFEF00D, 2**64 - 1])
def test_philox_matches_library_implementation(tmp_path, seed):
    """Oracle Philox4x32-10 == triton's tl.philox (an independent library
    implementation of the SC'11 generator, run on the CPU interpreter)."""
    rng = np.random.default_rng(seed % 2**32)
    ctrs = _edge_counters(rng, 600)
    np.savez(tmp_path / "in.npz", ctrs=ctrs, seed=np.uint64(seed))
    subprocess.run([sys.executable, os.path.join(HERE, "philox_library_ref.py"),
                    str(tmp_path / "in.npz"), str(tmp_path / "out.npy")], check=True,
                   timeout=600)
    ref = np.load(tmp_path / "out.npy")
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    got = oracle.philox(ctrs, key)
    assert np.array_equal(got, ref)


def test_sample_words_layout():
    """Dimension k of sample i takes word k mod 4 of the call with counter
    (i_lo, i_hi, floor(k/4) | id<<8, iteration) under key (seed_lo, seed_hi)."""
    seed, it, ident = 0x1234_5678_9ABC_DEF0, 7, 3
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    for i in [0, 1, 2**32 - 1, 2**32, 2**40 + 17]:
        for dim in [1, 3, 4, 5, 8, 16]:
            w = oracle.sample_words(seed, ident, it, i, dim)
            for k in range(dim):
                ctr = np.array([[i & 0xFFFFFFFF, i >> 32, (k // 4) | (ident << 8), it]],
                               dtype=np.uint32)
                assert w[k] == oracle.philox(ctr, key)[0, k % 4]


def test_philox_words_uniform():
    """Coarse uniformity: the top 8 bits of 2^18 words are flat (chi^2, 255 dof)."""
    n = 1 << 16
    ctrs = np.zeros((n, 4), dtype=np.uint32)
    ctrs[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle.philox(ctrs, np.array([42, 0], dtype=np.uint32)).ravel()
    counts = np.bincount(out >> 24, minlength=256)
    expect = out.size / 256
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert 150 < chi2 < 380
