"""The no-allocation entry point (vegas_iterate_noalloc) against the workspace
path (vegas_iterate + vegas_refine).

Some callers may not allocate device memory at all: code loaded into a host
framework that owns every device allocation, or code that only holds the
buffers it was handed.  vegas_iterate_noalloc serves them from a static device
array inside the library.  This file is collected last so that a run stopping
at the first failure has already run every other test; it also passes on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

RTOL = 1e-12  # the FP64 parity bound of the GPU tests
# FP32-eval: the float shared-memory histogram is summed in an order that
# differs from run to run, so two runs' refined grids differ at ~1e-7; the
# float tolerance of the parity tests applies (1e-5 on I, 10x on var)
RTOL32 = 1e-5


def _refined_tol(edges):
    # after a refinement both paths' edges agree to about an ulp (histogram
    # atomics add in different orders); J = prod N Delta turns that into
    # 8 d eps / min(Delta) on I, as in the parity tests
    dmin = np.min(np.diff(edges, axis=1))
    return max(RTOL, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def test_noalloc_rejects_a_histogram_larger_than_its_scratch():
    """dim * nbins above the static scratch's capacity is refused before any
    device work."""
    V.lib()
    p = (ctypes.c_double * 17)(*([0.1] + [0.5] * 16))
    out = V.lib().vegas_iterate_noalloc(ctypes.c_void_p(0x10000), 16, 257, 1, 0, 0, p, 17,
                                        1000, 1, 1.5, ctypes.c_void_p(0x20000), None)
    assert out == V.VEGAS_ENOSPACE
    assert V.vegas_strerror(out) == "workspace too small"


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_noalloc_matches_workspace_path_two_calls(mode):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    dim, nbins, seed, n, alpha = 4, 50, 11, 1_000_000, 1.5
    p = W.gauss_params(dim, 0.1, [0.5, 0.4, 0.6, 0.5])

    # the workspace path: two adapting iterations
    v = V.Vegas(dim, nbins, seed, mode, V.VEGAS_GAUSS, p, max_iters=4)
    grids = [v.grid()]
    for _ in range(2):
        v.iterate(n, 1)
        v.refine(alpha)
        grids.append(v.grid())
    rows = v.iterations()
    v.close()

    # the no-allocation path: the same two iterations, grid and result in
    # caller-owned device buffers
    stream = torch.cuda.current_stream()
    edges = torch.tensor(grids[0], dtype=torch.float64, device="cuda").contiguous()
    result = torch.zeros(6, dtype=torch.float64, device="cuda")
    for it in range(2):
        result.fill_(-1.0)
        V.vegas_iterate_noalloc(edges.data_ptr(), dim, nbins, seed, it, mode, p, n, 1, alpha,
                                result.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = result.cpu().numpy()
        ref = rows[it]
        if mode == V.VEGAS_FP32_EVAL:
            tol, edge_rtol, edge_atol = (RTOL if it == 0 else RTOL32), 0.0, 1e-6
        else:
            tol = RTOL if it == 0 else _refined_tol(grids[it])
            edge_rtol, edge_atol = RTOL, 1e-15  # the grid bound of the parity tests
        assert got[2] == n and got[3] == ref[3] == 0
        assert abs(got[4] - ref[4]) <= tol * abs(ref[4]), (it, got[4], ref[4], tol)
        assert abs(got[5] - ref[5]) <= (10 if mode else 100) * tol * ref[5], (it, got[5], ref[5])
        assert abs(got[0] - ref[0]) <= tol * abs(ref[0])
        assert np.allclose(edges.cpu().numpy(), grids[it + 1], rtol=edge_rtol,
                           atol=edge_atol), it
