"""The device refinement (vegas_refine) against the oracle's, one step, on
histograms chosen to reach its edge cases: installed into a state with
vegas_shard_import on a random monotone grid, refined once, compared with
oracle.refine on the same grid and histogram.  FP64 on both sides: 1e-12
relative, or the bound that summation order sets where a damped weight is
tiny (edge_tolerance)."""
import numpy as np
import pytest

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


def histograms(dim, nbins, rng):
    """Rows: smooth positive, a single hot bin, zeros with a few spikes, 30
    decades of dynamic range, first/last bin only, all zero (kept grid)."""
    rows = [rng.uniform(0.5, 2.0, nbins)]
    one = np.zeros(nbins)
    one[rng.integers(nbins)] = 3.0
    rows.append(one)
    sp = np.zeros(nbins)
    sp[rng.choice(nbins, size=max(1, nbins // 7), replace=False)] = rng.uniform(1, 10)
    rows.append(sp)
    rows.append(10.0 ** rng.uniform(-30, 0, nbins))
    ends = np.zeros(nbins)
    ends[0], ends[-1] = 1.0, 1e-3
    rows.append(ends)
    rows.append(np.zeros(nbins))
    return np.stack([rows[k % len(rows)] for k in range(dim)])


def refine_on_gpu(mode, edges, hist, alpha):
    dim, nb1 = edges.shape
    v = V.Vegas(dim, nb1 - 1, 1, mode, W.GAUSS, W.gauss_params(dim, 0.2), max_iters=4)
    v.set_grid(edges)
    from paper_2002_12921_b300.shard import GpuShardEngine

    eng = GpuShardEngine(v)
    eng.iterate_range(1000, 0, 1000, True)  # an adapting iteration, then install `hist`
    buf = torch.zeros(3 + hist.size, dtype=torch.float64, device="cuda")
    buf[0], buf[1] = 1.0, 1.0
    buf[3:] = torch.from_numpy(hist.reshape(-1)).cuda()
    eng.import_(buf, 1000)
    v.refine(alpha)
    out, h_after = v.grid(), v.histogram()
    v.close()
    return out, h_after


def edge_tolerance(edges, hist, alpha):
    """Per row, the absolute edge tolerance: a refined edge is
    e_b + (target - C_b) / m_b * Delta_b, and the cumulative sums C (warp scan
    on the device, sequential in the oracle) differ by a few eps * sum(m), so
    the edge moves by up to ~eps * sum(m) / m_b * Delta_b; bound it with the
    smallest positive damped weight and the widest bin, times 16."""
    eps = np.finfo(float).eps
    tol = np.zeros(edges.shape[0])
    for k in range(edges.shape[0]):
        sm = oracle.smooth(hist[k])
        if not sm.sum() > 0:
            continue                              # the row keeps its grid exactly
        m = np.array([oracle.damp(x, alpha) for x in sm / sm.sum()])
        tol[k] = 16 * eps * m.sum() / m[m > 0].min() * np.max(np.diff(edges[k]))
    return tol


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
@pytest.mark.parametrize("alpha", [0.0, 0.5, 1.5, 3.0])
@pytest.mark.parametrize("dim,nbins", [(6, 2), (6, 37), (6, 50), (12, 333), (3, 1024)])
def test_refine_matches_oracle_on_edge_case_histograms(mode, alpha, dim, nbins):
    rng = np.random.Generator(np.random.PCG64(dim * 1000 + nbins))
    edges = W.random_monotone_grid(dim, nbins, seed=nbins, spread=1.0)
    hist = histograms(dim, nbins, rng)
    got, h_after = refine_on_gpu(mode, edges, hist, alpha)
    ref = oracle.refine(edges, hist, alpha)
    tol = np.maximum(edge_tolerance(edges, hist, alpha)[:, None], 1e-12 * np.abs(ref)) + 1e-15
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)
    assert np.all(np.diff(got, axis=1) > 0) and np.all(got[:, 0] == 0) and np.all(got[:, -1] == 1)
    assert np.all(h_after == 0)                      # the histogram is cleared
    zero_rows = np.where(hist.sum(axis=1) == 0)[0]
    assert np.array_equal(got[zero_rows], edges[zero_rows])  # kept grid
