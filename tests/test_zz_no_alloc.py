"""The no-allocation entry point (vegas_iterate_noalloc) against the FP64 CPU
oracle and against the workspace path (vegas_iterate + vegas_refine).

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

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

from tests.fp32_budget import fp32_hist_tol, refine_edge_tol

RTOL = 1e-12  # the FP64 parity bound of the GPU tests
# FP32-eval on one grid and the same counters: the float budget of I for
# d <= 8 (10x on var), as in the parity tests
RTOL32 = 1e-5
DIM, NBINS, SEED, N, ALPHA = 4, 50, 11, 1_000_000, 1.5
MU = [0.5, 0.4, 0.6, 0.5]


def _refined_tol(edges):
    # after a refinement both paths' edges agree to about an ulp (histogram
    # atomics add in different orders); J = prod N Delta turns that into
    # 8 d eps / min(Delta) on I, as in the parity tests
    dmin = np.min(np.diff(edges, axis=1))
    return max(RTOL, 8 * edges.shape[0] * np.finfo(float).eps / dmin)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    return torch


def _noalloc(torch, edges, it, mode, p, n, adapt):
    """One call on the caller's device buffers; returns (result row, edges after)."""
    result = torch.full((6,), -1.0, dtype=torch.float64, device="cuda")
    V.vegas_iterate_noalloc(edges.data_ptr(), DIM, NBINS, SEED, it, mode, p, n, adapt, ALPHA,
                            result.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return result.cpu().numpy(), edges.cpu().numpy()


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
def test_noalloc_matches_oracle_and_workspace_path_two_calls(mode):
    """Two adapting calls in a row, then a fixed-grid call, on caller-owned
    device buffers.  Each adapting call's result row equals the oracle's
    iteration on the same grid and counters (FP64 1e-12; FP32 the float budget)
    and the grid it leaves equals the oracle's refinement (FP64 1e-12; FP32
    within what the float histogram budget lets a refinement move); each row and
    grid also equals the workspace path's.  The fixed-grid call (adapt = 0)
    equals the oracle's and the workspace path's fixed-grid iteration and
    leaves the grid bit for bit unchanged."""
    torch = _cuda()
    p = W.gauss_params(DIM, 0.1, MU)

    # the workspace path: two adapting iterations and one on the frozen grid
    v = V.Vegas(DIM, NBINS, SEED, mode, V.VEGAS_GAUSS, p, max_iters=4)
    grids = [v.grid()]
    for _ in range(2):
        v.iterate(N, 1)
        v.refine(ALPHA)
        grids.append(v.grid())
    v.iterate(N, 0)
    rows = v.iterations()
    v.close()

    edges = torch.tensor(oracle.uniform_grid(DIM, NBINS), dtype=torch.float64,
                         device="cuda").contiguous()
    for it in range(2):
        before = edges.cpu().numpy()
        got, after = _noalloc(torch, edges, it, mode, p, N, 1)
        o = oracle.iterate(before, SEED, it, N, W.GAUSS, p, True, nthreads=4)
        ref = rows[it]
        assert got[2] == N and got[3] == o["nonfinite"] == ref[3] == 0
        if mode == V.VEGAS_FP64:
            otol = RTOL
            wtol = RTOL if it == 0 else _refined_tol(grids[it])
            ref_grid = oracle.refine(before, o["hist"], ALPHA)
            assert np.allclose(after, ref_grid, rtol=RTOL, atol=1e-15), it
            assert np.allclose(after, grids[it + 1], rtol=RTOL, atol=1e-15), it
        else:
            # no pre-scale in this call (h = 0): the bin budget of fp32_budget
            otol = wtol = RTOL32
            rt, _ = fp32_hist_tol(W.GAUSS, DIM, p, before, N)
            etol = refine_edge_tol(before, o["hist"], ALPHA, rt)
            assert np.allclose(after, oracle.refine(before, o["hist"], ALPHA), rtol=0,
                               atol=etol), it
            # two float histograms summed in different orders: ~1e-7 apart
            assert np.allclose(after, grids[it + 1], rtol=0, atol=1e-6), it
        assert abs(got[4] - o["I"]) <= otol * abs(o["I"]), (it, got[4], o["I"])
        assert abs(got[5] - o["var"]) <= 10 * otol * (o["var"] + o["I"] ** 2 / N), it
        assert abs(got[0] - o["S1"]) <= otol * abs(o["S1"])
        if it == 0 or mode == V.VEGAS_FP32_EVAL:
            # the same grid on both paths (FP32: to the float histogram's order)
            assert abs(got[4] - ref[4]) <= wtol * abs(ref[4]), (it, got[4], ref[4])
            assert abs(got[5] - ref[5]) <= 10 * wtol * ref[5], (it, got[5], ref[5])
        else:
            assert abs(got[4] - ref[4]) <= wtol * abs(ref[4]), (it, got[4], ref[4])
            assert abs(got[5] - ref[5]) <= 100 * wtol * ref[5], (it, got[5], ref[5])

    # a fixed-grid call: the grid is left exactly as it was
    before = edges.cpu().numpy()
    got, after = _noalloc(torch, edges, 2, mode, p, N, 0)
    assert np.array_equal(after, before)
    o = oracle.iterate(before, SEED, 2, N, W.GAUSS, p, False, nthreads=4)
    tol = RTOL if mode == V.VEGAS_FP64 else RTOL32
    assert got[2] == N and got[3] == 0
    assert abs(got[4] - o["I"]) <= tol * abs(o["I"]), (got[4], o["I"])
    assert abs(got[5] - o["var"]) <= 10 * tol * (o["var"] + o["I"] ** 2 / N)
    # the workspace path ran its fixed-grid iteration on its own refined grid
    wtol = _refined_tol(grids[2]) if mode == V.VEGAS_FP64 else RTOL32
    assert abs(got[4] - rows[2][4]) <= wtol * abs(rows[2][4]), (got[4], rows[2][4])


@pytest.mark.gpu
def test_noalloc_fixed_grid_then_adapting_call():
    """A fixed-grid call leaves the scratch's ticket ready for the next call: an
    adapting call right after it equals the oracle's iteration and refinement."""
    torch = _cuda()
    p = W.gauss_params(DIM, 0.1, MU)
    edges = torch.tensor(oracle.uniform_grid(DIM, NBINS), dtype=torch.float64,
                         device="cuda").contiguous()
    got0, _ = _noalloc(torch, edges, 0, V.VEGAS_FP64, p, 200_000, 0)
    got1, after = _noalloc(torch, edges, 1, V.VEGAS_FP64, p, 200_000, 1)
    e = oracle.uniform_grid(DIM, NBINS)
    o0 = oracle.iterate(e, SEED, 0, 200_000, W.GAUSS, p, False)
    o1 = oracle.iterate(e, SEED, 1, 200_000, W.GAUSS, p, True)
    assert abs(got0[4] - o0["I"]) <= RTOL * abs(o0["I"])
    assert abs(got1[4] - o1["I"]) <= RTOL * abs(o1["I"])
    assert np.allclose(after, oracle.refine(e, o1["hist"], ALPHA), rtol=RTOL, atol=1e-15)


@pytest.mark.gpu
def test_noalloc_refuses_a_host_result_pointer():
    """d_result must be device memory on the grid's device: a host buffer is
    refused with VEGAS_EINVAL before anything is enqueued, and the grid is left
    untouched."""
    torch = _cuda()
    p = W.gauss_params(DIM, 0.1, MU)
    edges = torch.tensor(oracle.uniform_grid(DIM, NBINS), dtype=torch.float64,
                         device="cuda").contiguous()
    host = np.zeros(6)
    pp = (ctypes.c_double * len(p))(*p)
    rc = V.lib().vegas_iterate_noalloc(ctypes.c_void_p(edges.data_ptr()), DIM, NBINS, SEED, 0,
                                       V.VEGAS_FP64, pp, len(p), 10_000, 1, ALPHA,
                                       ctypes.c_void_p(host.ctypes.data),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == V.VEGAS_EINVAL
    assert np.array_equal(edges.cpu().numpy(), oracle.uniform_grid(DIM, NBINS))
    assert np.all(host == 0.0)
