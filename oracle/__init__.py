"""FP64 CPU oracle of the Vegas iteration (test infrastructure).

This package is test infrastructure.  Only the test suite, the smoke check and
the benchmark's CPU-baseline / reference leg may import it.  It shares no code
with the CUDA library: it wraps the plain C restatement in ``vegas_oracle.c``
(compiled by ``build_oracle.py``) with ctypes, and adds the Python-level driver
loop (iterate, then refine) that the paper's two integrator hooks describe
(VegasFlow Sec. 2.2: a per-event step, then an after-iteration refinement).
"""
import ctypes
import os

import numpy as np

from .build_oracle import build as _build

GAUSS, GAUSS_MIX2, FLAT, GENZ_DISC, GENZ_PPEAK = 0, 1, 2, 3, 4

_lib = None


def lib():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        # VEGAS_ORACLE_LIBRARY: another build of the oracle (the test suite's
        # planted-mistake check points it at altered copies)
        path = os.environ.get("VEGAS_ORACLE_LIBRARY") or _build()
        L = ctypes.CDLL(path)
        u64, i32, u32, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
        vp = ctypes.c_void_p
        L.oracle_philox_batch.argtypes = [u64, vp, vp, vp]
        L.oracle_philox_batch.restype = None
        L.oracle_sample_words.argtypes = [u64, u32, u32, u64, i32, vp]
        L.oracle_sample_words.restype = None
        L.oracle_map_batch.argtypes = [u64, i32, i32, vp, vp, vp, vp, vp]
        L.oracle_map_batch.restype = None
        L.oracle_integrand_batch.argtypes = [u64, i32, i32, vp, vp, vp]
        L.oracle_integrand_batch.restype = None
        L.oracle_iterate.argtypes = [i32, i32, vp, u64, u32, u32, u64, i32, vp, i32, i32,
                                     vp, vp, vp, vp]
        L.oracle_iterate.restype = i32
        L.oracle_iterate_range.argtypes = [i32, i32, vp, u64, u32, u32, u64, u64, i32, vp, i32,
                                           i32, vp, vp, vp, vp]
        L.oracle_iterate_range.restype = i32
        L.oracle_iterate_range_box.argtypes = [i32, i32, vp, u64, u32, u32, u64, u64, i32, vp,
                                               vp, vp, i32, i32, vp, vp, vp, vp]
        L.oracle_iterate_range_box.restype = i32
        L.oracle_estimate.argtypes = [dbl, dbl, u64, vp, vp]
        L.oracle_estimate.restype = None
        L.oracle_damp.argtypes = [dbl, dbl]
        L.oracle_damp.restype = dbl
        L.oracle_smooth.argtypes = [i32, vp, vp]
        L.oracle_smooth.restype = None
        L.oracle_refine.argtypes = [i32, i32, vp, vp, dbl]
        L.oracle_refine.restype = i32
        L.oracle_combine.argtypes = [i32, vp, vp, vp, vp, vp]
        L.oracle_combine.restype = None
        L.oracle_gauss_gradient.argtypes = [i32, i32, vp, u64, u32, u64, vp, vp]
        L.oracle_gauss_gradient.restype = i32
        L.oracle_gauss_gradient_box.argtypes = [i32, i32, vp, u64, u32, u64, vp, vp, vp, vp]
        L.oracle_gauss_gradient_box.restype = i32
        L.oracle_uniform_grid.argtypes = [i32, i32, vp]
        L.oracle_uniform_grid.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def philox(ctrs, key):
    """Philox4x32-10 of each counter row (n x 4 uint32) under key (2 uint32)."""
    ctrs = _c(ctrs, np.uint32).reshape(-1, 4)
    key = _c(key, np.uint32).reshape(2)
    out = np.empty_like(ctrs)
    lib().oracle_philox_batch(ctrs.shape[0], _ptr(ctrs), _ptr(key), _ptr(out))
    return out


def sample_words(seed, integral_id, it, i, dim):
    """The dim Philox words of sample i in iteration it."""
    w = np.empty(dim, dtype=np.uint32)
    lib().oracle_sample_words(seed, integral_id, it, i, dim, _ptr(w))
    return w


def uniform_grid(dim, nbins):
    e = np.empty((dim, nbins + 1), dtype=np.float64)
    lib().oracle_uniform_grid(dim, nbins, _ptr(e))
    return e


def map_samples(edges, words):
    """Grid map of word rows (n x d): returns x (n x d), J (n), bins (n x d)."""
    edges = _c(edges, np.float64)
    dim, nb1 = edges.shape
    words = _c(words, np.uint32).reshape(-1, dim)
    n = words.shape[0]
    x = np.empty((n, dim))
    J = np.empty(n)
    bins = np.empty((n, dim), dtype=np.int32)
    lib().oracle_map_batch(n, dim, nb1 - 1, _ptr(edges), _ptr(words), _ptr(x), _ptr(J), _ptr(bins))
    return x, J, bins


def integrand(fid, params, x):
    """Integrand fid at points x (n x d)."""
    x = _c(x, np.float64)
    n, dim = x.shape
    p = _c(params if params is not None and len(params) else [0.0], np.float64)
    f = np.empty(n)
    lib().oracle_integrand_batch(n, fid, dim, _ptr(p), _ptr(x), _ptr(f))
    return f


def _box(box, dim):
    """(lo, w) arrays for a box [(lo_k, hi_k)] or (None, None) for the unit cube."""
    if box is None:
        return None, None
    b = np.asarray(box, dtype=np.float64).reshape(dim, 2)
    return _c(b[:, 0], np.float64), _c(b[:, 1] - b[:, 0], np.float64)


def iterate(edges, seed, it, n, fid, params, adapt, integral_id=0, nthreads=1, box=None):
    """One iteration: returns dict(S1, S2, nonfinite, hist (d x N) or None, I, var).
    box: [(lo_k, hi_k)] per dimension (None: the unit cube)."""
    edges = _c(edges, np.float64)
    dim, nb1 = edges.shape
    nbins = nb1 - 1
    p = _c(params if params is not None and len(params) else [0.0], np.float64)
    hist = np.zeros((dim, nbins)) if adapt else None
    S1 = np.zeros(1)
    S2 = np.zeros(1)
    bad = np.zeros(1, dtype=np.uint64)
    lo, w = _box(box, dim)
    rc = lib().oracle_iterate_range_box(dim, nbins, _ptr(edges), seed, integral_id, it, 0, n,
                                        fid, _ptr(p), _ptr(lo), _ptr(w), 1 if adapt else 0,
                                        nthreads, _ptr(S1), _ptr(S2), _ptr(hist), _ptr(bad))
    if rc != 0:
        raise ValueError("oracle_iterate: invalid arguments")
    I, var = estimate(S1[0], S2[0], n)
    return dict(S1=float(S1[0]), S2=float(S2[0]), nonfinite=int(bad[0]), hist=hist, I=I, var=var)


def iterate_range(edges, seed, it, first, count, fid, params, adapt, integral_id=0, nthreads=1):
    """Partial sums of samples [first, first+count) of iteration it: dict(S1, S2,
    nonfinite, hist (d x N) or None)."""
    edges = _c(edges, np.float64)
    dim, nb1 = edges.shape
    p = _c(params if params is not None and len(params) else [0.0], np.float64)
    hist = np.zeros((dim, nb1 - 1)) if adapt else None
    S1, S2 = np.zeros(1), np.zeros(1)
    bad = np.zeros(1, dtype=np.uint64)
    if lib().oracle_iterate_range(dim, nb1 - 1, _ptr(edges), seed, integral_id, it, first, count,
                                  fid, _ptr(p), 1 if adapt else 0, nthreads, _ptr(S1), _ptr(S2),
                                  _ptr(hist), _ptr(bad)):
        raise ValueError("oracle_iterate_range: invalid arguments")
    return dict(S1=float(S1[0]), S2=float(S2[0]), nonfinite=int(bad[0]), hist=hist)


def estimate(S1, S2, n):
    I = np.zeros(1)
    v = np.zeros(1)
    lib().oracle_estimate(S1, S2, n, _ptr(I), _ptr(v))
    return float(I[0]), float(v[0])


def damp(r, alpha):
    return lib().oracle_damp(float(r), float(alpha))


def smooth(row):
    """Three-point smoothing of one histogram row."""
    row = _c(row, np.float64)
    out = np.empty_like(row)
    lib().oracle_smooth(len(row), _ptr(row), _ptr(out))
    return out


def refine(edges, hist, alpha):
    """Refined copy of edges (d x (N+1)) from hist (d x N)."""
    e = _c(edges, np.float64).copy()
    h = _c(hist, np.float64)
    lib().oracle_refine(e.shape[0], e.shape[1] - 1, _ptr(e), _ptr(h), float(alpha))
    return e


def combine(I, var):
    """Inverse-variance combination: (mean, sigma, chi2/dof)."""
    I = _c(I, np.float64)
    var = _c(var, np.float64)
    out = np.zeros(3)
    lib().oracle_combine(len(I), _ptr(I), _ptr(var), _ptr(out[0:]), _ptr(out[1:]), _ptr(out[2:]))
    return float(out[0]), float(out[1]), float(out[2])


def gauss_gradient(edges, seed, it, n, params, box=None):
    """Fixed-grid estimate of the Eq. 1 integral and its gradient in
    (mu_1..mu_d, a) over samples 0..n-1 of iteration it: dict(I, dmu, da,
    var_I, var_dmu, var_da, nonfinite).  box: [(lo_k, hi_k)] per dimension
    (None: the unit cube)."""
    edges = _c(edges, np.float64)
    dim, nb1 = edges.shape
    p = _c(params, np.float64)
    out = np.zeros(2 * (dim + 2) + 1)
    lo, w = _box(box, dim)
    if lib().oracle_gauss_gradient_box(dim, nb1 - 1, _ptr(edges), seed, it, n, _ptr(p), _ptr(lo),
                                       _ptr(w), _ptr(out)):
        raise ValueError("oracle_gauss_gradient: invalid arguments")
    nc = dim + 2
    return dict(I=out[0], dmu=out[1:dim + 1].copy(), da=out[dim + 1], var_I=out[nc],
                var_dmu=out[nc + 1:nc + 1 + dim].copy(), var_da=out[nc + dim + 1],
                nonfinite=int(out[2 * nc]), raw=out)


def run(dim, nbins, seed, fid, params, schedule, alpha=1.5, integral_id=0, nthreads=1,
        edges=None, first_iter=0, box=None):
    """A whole Vegas run.  schedule: list of (n_samples, adapt) per iteration.
    Each adapting iteration is followed by a refinement of the grid.
    Returns dict(log=[iteration dicts], edges=final grid, grids=[grid used per
    iteration], mean, sigma, chi2_dof over iterations >= first_iter)."""
    e = uniform_grid(dim, nbins) if edges is None else _c(edges, np.float64).copy()
    log, grids = [], []
    for it, (n, adapt) in enumerate(schedule):
        grids.append(e.copy())
        r = iterate(e, seed, it, n, fid, params, adapt, integral_id, nthreads, box)
        r["n"] = n
        log.append(r)
        if adapt:
            e = refine(e, r["hist"], alpha)
    sel = log[first_iter:]
    mean, sigma, chi2 = combine([r["I"] for r in sel], [r["var"] for r in sel])
    return dict(log=log, edges=e, grids=grids, mean=mean, sigma=sigma, chi2_dof=chi2)
