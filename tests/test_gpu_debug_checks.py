"""The debug build's device checks (libvegas_b300_debug.so, VEGAS_DEBUG_CHECKS):
valid runs pass every check in both precisions and in a batch, and a grid
corrupted in device memory (two edges swapped, bypassing vegas_set_grid's
validation) is reported by vegas_result as VEGAS_ESTATE.  A corrupted grid only
changes arithmetic -- edges never form addresses -- so the run itself is safe.
The checks run in a child process that loads the debug library."""
import os
import subprocess
import sys

import pytest

from paper_2002_12921_b300 import build

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

assert V.binding.LIB_PATH.endswith("libvegas_b300_debug.so"), V.binding.LIB_PATH
for mode in (V.VEGAS_FP64, V.VEGAS_FP32_EVAL):
    v = V.Vegas(4, 20, 3, mode, V.VEGAS_GAUSS, W.gauss_params(4, 0.2), max_iters=8)
    v.run([(100_000, 1)] * 3 + [(100_000, 0)])
    mean = v.result(0)[0]          # raises if a check failed
    assert abs(mean - 0.9984) < 0.01, mean
    # swap two interior edges of dimension 2 in device memory (the edges are the
    # first dim x (nbins + 1) doubles of the workspace)
    e = v.grid()
    e[2, 5], e[2, 6] = e[2, 6], e[2, 5]
    v.workspace[: e.size * 8].copy_(torch.from_numpy(e.reshape(-1).copy().view(np.uint8)))
    v.iterate(50_000, 0)
    try:
        v.result(0)
    except V.VegasError as exc:
        assert exc.status == V.VEGAS_ESTATE, exc.status
    else:
        raise AssertionError("corrupted grid not reported (mode %d)" % mode)
    v.close()

dims, ns = [2, 7, 12], [5000, 20000, 9000]
params = [W.gauss_params(d, 0.2) for d in dims]
B = V.VegasBatch(dims, ns, 25, 5, V.VEGAS_FP32_EVAL, params, max_iters=4)
B.run(3)
for b in range(3):
    B.result(b)                    # raises if a check failed
B.close()
print("debug checks: ok")
'''


def test_debug_build_checks_pass_valid_runs_and_catch_a_corrupted_grid():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lib = build.build(debug=True)
    env = dict(os.environ, VEGAS_B300_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "debug checks: ok" in r.stdout
