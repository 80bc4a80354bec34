"""Seeded synthetic workloads for the Vegas hot path.

This module only describes inputs: dimensions, bin counts, iteration schedules
and integrand parameters drawn from seeded numpy generators.  It holds none of
the method's arithmetic (no map, no integrand evaluation, no refinement, no
normalisation constants), so that both the CUDA path and the CPU oracle can be
fed the same inputs without sharing code.

The integrands are the paper's toy functions over [0,1]^d (VegasFlow Sec. 3.1,
Eq. 1-3); the paper names no dataset, so seeded parameters stand in for its
choices, which it does not print.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# integrand ids, the same numbering as the C ABI's vegas_integrand
GAUSS, GAUSS_MIX2, FLAT, GENZ_DISC, GENZ_PPEAK = 0, 1, 2, 3, 4


@dataclass
class Workload:
    name: str
    dim: int
    nbins: int
    integrand: int
    params: List[float]
    schedule: List[Tuple[int, int]]  # (samples, adapt) per iteration
    seed: int
    alpha: float = 1.5
    first_iter: int = 0  # first iteration entering the combined result
    chunk: int = 0  # samples per launch (0: one launch per iteration)
    notes: str = field(default="")

    @property
    def total_samples(self) -> int:
        return int(sum(n for n, _ in self.schedule))


def gauss_params(dim: int, a: float, mu=0.5) -> List[float]:
    """[a, mu_1..mu_d] for the Lepage Gaussian of Eq. 1."""
    mu = np.broadcast_to(np.asarray(mu, dtype=np.float64), (dim,))
    return [float(a)] + [float(m) for m in mu]


def mix2_params(dim: int, a: float, c1: float = 1.0 / 3.0, c2: float = 2.0 / 3.0) -> List[float]:
    """[a, muA_1..muA_d, muB_1..muB_d] for the two-peak mixture."""
    return [float(a)] + [float(c1)] * dim + [float(c2)] * dim


def c1_gauss4(seed: int = 1) -> Workload:
    """d=4 Lepage Gaussian, a=0.1, 50 bins, 5 adapting iterations of 1e5."""
    return Workload("gauss_d4_a0.1_N50_5x1e5", 4, 50, GAUSS, gauss_params(4, 0.1),
                    [(100_000, 1)] * 5, seed)


def c2_gauss8(seed: int = 2, n_adapt: int = 10_000_000, n_fixed: int = 100_000_000,
              it_adapt: int = 10, it_fixed: int = 5) -> Workload:
    """d=8 Lepage Gaussian, a=0.1, 50 bins: 10 adapting iterations of 1e7, then
    5 fixed-grid iterations of 1e8; the result combines the fixed-grid ones."""
    return Workload(f"gauss_d8_a0.1_N50_{it_adapt}x{n_adapt:.0e}+{it_fixed}x{n_fixed:.0e}",
                    8, 50, GAUSS, gauss_params(8, 0.1),
                    [(n_adapt, 1)] * it_adapt + [(n_fixed, 0)] * it_fixed, seed,
                    first_iter=it_adapt)


def c3_centres(seed: int = 3, dim: int = 8) -> np.ndarray:
    """Per-dimension centres mu_i ~ U(0.3, 0.7) from numpy's PCG64."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(0.3, 0.7, size=dim)


def c3_gauss8_grad(seed: int = 3, n_warm: int = 1_000_000, n: int = 100_000_000) -> Workload:
    """d=8 Gaussian, width a=0.15, centres from c3_centres: 5 warm-up adapting
    iterations, then one fixed-grid iteration of n samples for I and dI/dtheta."""
    return Workload("gauss_d8_a0.15_grad", 8, 50, GAUSS, gauss_params(8, 0.15, c3_centres(seed)),
                    [(n_warm, 1)] * 5 + [(n, 0)], seed, first_iter=5)


def c4_batch(seed: int = 4, count: int = 256, iters: int = 8) -> List[Workload]:
    """256 independent Gaussians: d ~ U{2..16}, samples/iteration log-uniform in
    [1e4, 1e6], a ~ U(0.05, 0.3), centres ~ U(0.2, 0.8), 50 bins, 8 adapting
    iterations each."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for b in range(count):
        d = int(rng.integers(2, 17))
        n = int(round(10 ** rng.uniform(4.0, 6.0)))
        a = float(rng.uniform(0.05, 0.3))
        mu = rng.uniform(0.2, 0.8, size=d)
        out.append(Workload(f"batch{b}", d, 50, GAUSS, gauss_params(d, a, mu),
                            [(n, 1)] * iters, seed))
    return out


def c5_mix16(seed: int = 5, n: int = 1_000_000_000, iters: int = 20,
             chunk: int = 100_000_000) -> Workload:
    """d=16 two-peak mixture (centres 1/3 and 2/3), a=0.1, 100 bins: 20
    adapting iterations of 1e9 samples streamed in 1e8-sample launches."""
    return Workload("mix2_d16_a0.1_N100", 16, 100, GAUSS_MIX2, mix2_params(16, 0.1),
                    [(n, 1)] * iters, seed, chunk=chunk)


def genz_params(dim: int, seed: int, kind: int) -> List[float]:
    """[a_1..a_d, c_1..c_d] for the Genz functions of Eq. 2 and Eq. 3.  The paper
    prints neither a_i nor c_i; these seeded draws stand in: thresholds a_i ~
    U(0.1, 0.4) and rates c_i ~ U(1, 3) for Eq. 2, centres a_i ~ U(0.3, 0.7) and
    sharpness c_i ~ U(5, 15) for Eq. 3."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if kind == GENZ_DISC:
        a = rng.uniform(0.1, 0.4, size=dim)
        c = rng.uniform(1.0, 3.0, size=dim)
    else:
        a = rng.uniform(0.3, 0.7, size=dim)
        c = rng.uniform(5.0, 15.0, size=dim)
    return [float(v) for v in a] + [float(v) for v in c]


def random_monotone_grid(dim: int, nbins: int, seed: int, spread: float = 1.0) -> np.ndarray:
    """A seeded strictly increasing grid per dimension with e_0 = 0, e_N = 1:
    bin widths proportional to exp(spread * z), z standard normal."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.exp(spread * rng.standard_normal((dim, nbins)))
    c = np.concatenate([np.zeros((dim, 1)), np.cumsum(w, axis=1)], axis=1)
    e = c / c[:, -1:]
    e[:, 0] = 0.0
    e[:, -1] = 1.0
    return e
