"""Float error budget of the FP32-eval path against the FP64 oracle (test helper).

The float path and the oracle draw the same Philox words, so every sample lands
in the same bins on both sides (the bin index is integer arithmetic); what
differs is the arithmetic of the map and the integrand, done in float on the
GPU.  This module bounds, from the grid and the integrand's parameters, how far
one sample's weight f J can move, and from that how far a bin of the (f J)^2
histogram of Lepage's refinement (1978 Sec. 3: the accumulator sum f^2 J^2 per
bin) can move.  The derivation (u = 2^-24, the float unit roundoff):

* staged coordinate z_k = sc_k x_k + sh_k: the float path stages each bin as
  (sc e' + sh, sc Delta), each rounded once, and forms z with one FMA from a
  23-bit fraction (the oracle uses 32 bits, so the two fractions differ by at
  most 2^-24 of the bin): |dz_k| <= u (3 zmax_k + 4 sc_k Delta_max,k), zmax_k
  the largest |z_k| over the box;
* Jacobian: d staged widths, ceil(d/4) exact N^4 factors and the prefactor,
  one rounding per product: (2 d + d/4 + 4) u;
* Eq. 1 Gaussian and the mixture, f = 2^-s with s = sum z_k^2 accumulated by
  FMAs: |ds| <= 2 sum |z_k||dz_k| + d u s, and sum |z_k||dz_k| <= sqrt(s) |dz|_2
  (Cauchy-Schwarz), then |d ln f| <= ln 2 |ds| + 4 u (ex2.approx);  s itself is
  capped at the largest value whose square still reaches float's range after
  the pre-scale (smaller contributions are below the absolute floor below);
* Eq. 3 product peak: |d ln f| <= sum_k (|dz_k| + 2 u) + 4 u, since
  2|z|/(1 + z^2) <= 1;
* Eq. 2 discontinuous: f = 2^(sum c'_k x_k), |d ln f| <= ln 2 (sum |c'_k| |dz_k|
  + d u sum |c'_k|) + 4 u (threshold decisions are compared in the same
  precision only up to this bound; a sample within ~1e-7 of a threshold could
  flip, which none of the seeded cases here does);
* one bin of the histogram: each (f J)^2 carries twice f J's bound plus one
  rounding, and a float copy sums m of them (m bounded from the launch shape)
  before the 32 copies are added in float and the bin goes to double:
  rtol = 2 d(fJ) + (m + 35) u;  absolute floor: every sample whose float
  (f J 2^-h)^2 falls below the smallest subnormal, 2^-149, is lost, so
  atol = n 2^-149 2^2h.
"""
import math

import numpy as np

import oracle

U = 2.0 ** -24
LN2 = math.log(2.0)
LOG2E = 1.0 / LN2
GAUSS, GAUSS_MIX2, FLAT, GENZ_DISC, GENZ_PPEAK = 0, 1, 2, 3, 4


def _staging(fid, dim, params):
    """(sc_k, centre lists) of the float staging z = sc (x - centre)."""
    p = np.asarray(params, dtype=np.float64)
    if fid in (GAUSS, GAUSS_MIX2):
        kappa = math.sqrt(LOG2E) / p[0]
        centres = [p[1:1 + dim]]
        if fid == GAUSS_MIX2:
            centres.append(p[1 + dim:1 + 2 * dim])
        return np.full(dim, kappa), centres
    if fid == GENZ_PPEAK:
        return p[dim:2 * dim].copy(), [p[:dim]]
    return np.ones(dim), [np.zeros(dim)]


def fp32_weight_rtol(fid, dim, params, edges, h=0):
    """Bound on the relative error of one sample's f J (float path vs oracle)
    on the grid `edges`; h is the float path's pre-scale exponent (the ilogb of
    the previous iteration's estimate, 0 on the first)."""
    edges = np.asarray(edges, dtype=np.float64)
    nbins = edges.shape[1] - 1
    dmax = np.max(np.diff(edges, axis=1), axis=1)
    sc, centres = _staging(fid, dim, params)
    jac = (2 * dim + dim / 4 + 4) * U
    if fid == FLAT:
        return jac + U
    dlnf = 0.0
    if fid in (GAUSS, GAUSS_MIX2):
        # largest s that still matters: (f J 2^-h)^2 >= 2^-149 needs
        # f >= 2^-75 / max(J C 2^-h), and J C = prod_k N Delta_k / (a sqrt(pi))
        a = float(params[0])
        log2_jc = float(np.sum(np.log2(nbins * dmax))) - dim * math.log2(a * math.sqrt(math.pi))
        s_cap = 75.0 + max(0.0, log2_jc - h) + 1.0
        for c in centres:
            zmax = sc * np.maximum(np.abs(c), np.abs(1.0 - c))
            dz = U * (3 * zmax + 4 * sc * dmax)
            s = min(float(np.sum(zmax ** 2)), s_cap)
            cross = min(float(np.sum(zmax * dz)), math.sqrt(s) * float(np.linalg.norm(dz)))
            dlnf = max(dlnf, LN2 * (2 * cross + dim * U * s) + 4 * U)
        if fid == GAUSS_MIX2:
            dlnf += U  # the sum of the two terms
    elif fid == GENZ_PPEAK:
        zmax = sc * np.maximum(np.abs(centres[0]), np.abs(1.0 - centres[0]))
        dz = U * (3 * zmax + 4 * sc * dmax)
        dlnf = float(np.sum(dz + 2 * U)) + 4 * U
    elif fid == GENZ_DISC:
        c2 = np.abs(np.asarray(params[dim:2 * dim], dtype=np.float64)) * LOG2E
        dz = U * (3.0 + 4 * dmax)
        dlnf = LN2 * (float(np.sum(c2 * dz)) + dim * U * float(np.sum(c2))) + 4 * U
    return dlnf + jac + U


def copy_adds_bound(n, nbins, copies=32, sms=148, block=256, min_per_thread=8):
    """Upper bound on the float additions one shared histogram copy makes into
    one bin in a launch of n samples: the launch has at least
    min(sms, ceil(n / (block min_per_thread))) blocks, each copy takes the
    samples of its lanes, and bins have probability 1/N (a 4-sigma allowance
    for the binomial count)."""
    blocks = max(1, min(sms, -(-n // (block * min_per_thread))))
    mean = n / (blocks * copies * nbins)
    return int(math.ceil(mean + 4 * math.sqrt(mean) + 4))


def fp32_hist_tol(fid, dim, params, edges, n, h=0, copies=32, **launch):
    """(rtol, atol) of one bin of the float path's (f J)^2 histogram against
    the oracle's, on the same grid and counters."""
    d = fp32_weight_rtol(fid, dim, params, edges, h)
    m = copy_adds_bound(n, np.asarray(edges).shape[1] - 1, copies, **launch)
    rtol = 2 * d + U + (m + 35) * U
    atol = n * 2.0 ** -149 * 2.0 ** (2 * h)
    return rtol, atol


def prescale_h(prev_estimate):
    """The float path's pre-scale exponent after an iteration whose estimate
    was prev_estimate: ilogb clamped to [-120, 120] (0 without one)."""
    if prev_estimate is None or not (prev_estimate > 0.0) or not math.isfinite(prev_estimate):
        return 0
    return max(-120, min(120, math.frexp(prev_estimate)[1] - 1))


def assert_hist_close(got, ref, rtol, atol, what=""):
    """Every bin within rtol of the oracle's (or within atol, the float floor),
    with the worst bin named in the failure message."""
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    assert got.shape == ref.shape, (what, got.shape, ref.shape)
    err = np.abs(got - ref)
    lim = rtol * np.abs(ref) + atol
    bad = err > lim
    if bad.any():
        k, j = np.unravel_index(int(np.argmax(err / lim)), got.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} bins outside rtol {rtol:.3g} / atol "
                             f"{atol:.3g}; worst bin ({k}, {j}): gpu {got[k, j]!r} oracle "
                             f"{ref[k, j]!r} rel {err[k, j] / max(abs(ref[k, j]), 1e-300):.3g}")
    return float(np.max(err / np.maximum(np.abs(ref), 1e-300), initial=0.0, where=ref > atol / rtol))


def refine_edge_tol(edges, hist, alpha, rtol, seed=0):
    """How far the refined grid may move when every bin of `hist` may be off by
    a relative rtol: twice the largest edge shift of the oracle's refinement
    under four such perturbations (two random sign patterns, and the two
    half-and-half patterns that shift the cumulative sums the most)."""
    hist = np.asarray(hist, dtype=np.float64)
    base = oracle.refine(edges, hist, alpha)
    nb = hist.shape[1]
    rng = np.random.default_rng(seed)
    half = np.where(np.arange(nb) < nb // 2, 1.0, -1.0)
    signs = [rng.choice([-1.0, 1.0], size=hist.shape), rng.choice([-1.0, 1.0], size=hist.shape),
             np.broadcast_to(half, hist.shape), np.broadcast_to(-half, hist.shape)]
    worst = 0.0
    for sg in signs:
        moved = oracle.refine(edges, hist * (1.0 + rtol * sg), alpha)
        worst = max(worst, float(np.max(np.abs(moved - base))))
    return 2.0 * worst + 1e-15
