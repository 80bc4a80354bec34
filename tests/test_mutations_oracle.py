"""The oracle's pins catch plausible mistakes (CPU only).

Each entry below plants one mistake in a copy of oracle/vegas_oracle.c -- a
wrong constant, a dropped factor, a swapped word or operand, an off-by-one, a
wrong divisor -- compiles the copy with the oracle's own flags, and runs the
oracle pin suite (tests/test_oracle_*.py) against it through
VEGAS_ORACLE_LIBRARY.  Every mutant must make at least one pin fail.  The
unaltered source is first run through the same harness and must pass, so a
broken harness cannot pass as a catch."""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import build_oracle  # noqa: E402

SRC = os.path.join(ROOT, "oracle", "vegas_oracle.c")
PINS = sorted(glob.glob(os.path.join(ROOT, "tests", "test_oracle_*.py")))

# (name, text in vegas_oracle.c, replacement): each text occurs exactly once
MUTANTS = [
    # Philox4x32-10
    ("philox multiplier", "PHILOX_M0 = 0xD2511F53u", "PHILOX_M0 = 0xD2511F35u"),
    ("philox key schedule", "k0 += PHILOX_W0;", "k0 += PHILOX_W1;"),
    ("philox word swap", "uint32_t y1 = lo1;", "uint32_t y1 = hi1;"),
    ("counter without the iteration", "ctr[3] = iter;", "ctr[3] = 0;"),
    ("counter integral shift", "ctr[2] = q | (integral_id << 8);",
     "ctr[2] = q | (integral_id << 4);"),
    ("word order", "words[4 * q + w] = out[w];", "words[4 * q + w] = out[3 - w];"),
    # bin, fraction, map, Jacobian
    ("fraction without the half", "double frac = ((double)l + 0.5) * 0x1p-32;",
     "double frac = ((double)l) * 0x1p-32;"),
    ("mirrored map", "x[k] = e[j] + frac * width;", "x[k] = e[j + 1] - frac * width;"),
    ("Jacobian without N", "J = J * ((double)nbins * width);", "J = J * width;"),
    # integrands
    ("Gaussian normalisation", "pow(a * sqrt(M_PI), -(double)dim)",
     "pow(a * sqrt(2.0 * M_PI), -(double)dim)"),
    ("Gaussian exponent", "return norm * exp(-s / (a * a));", "return norm * exp(-s / a);"),
    ("mixture second centre", "gauss_product(dim, params[0], params + 1 + dim, x)",
     "gauss_product(dim, params[0], params + dim, x)"),
    ("Genz discontinuity side", "if (x[k] <= a[k]) return 0.0;",
     "if (x[k] >= a[k]) return 0.0;"),
    ("Genz product-peak width", "double factor = 1.0 / (1.0 / (c[k] * c[k]) + u * u);",
     "double factor = 1.0 / (1.0 / c[k] + u * u);"),
    # sums and estimate
    ("histogram of f J, not (f J)^2", "jb->hist[(size_t)k * jb->nbins + bins[k]] += fw2;",
     "jb->hist[(size_t)k * jb->nbins + bins[k]] += fw;"),
    ("variance divisor n", "double v = (S2 / nn - (*I) * (*I)) / (nn - 1.0);",
     "double v = (S2 / nn - (*I) * (*I)) / nn;"),
    # refinement
    ("smoothing end weight", "out[0] = (hist[0] + hist[1]) / 2.0;",
     "out[0] = (hist[0] + hist[1]) / 3.0;"),
    ("smoothing interior weights", "(hist[j - 1] + hist[j] + hist[j + 1]) / 3.0",
     "(hist[j - 1] + 2.0 * hist[j] + hist[j + 1]) / 4.0"),
    ("damping exponent", "return pow((r - 1.0) / log(r), alpha);",
     "return pow((r - 1.0) / log(r), 1.0 / alpha);"),
    ("damping without normalisation", "m[j] = oracle_damp(sm[j] / smsum, alpha);",
     "m[j] = oracle_damp(sm[j], alpha);"),
    ("search tie to the upper bin", "while (b < N - 1 && !(target <= C[b + 1])) ++b;",
     "while (b < N - 1 && !(target < C[b + 1])) ++b;"),
    ("interpolation by m, not 1/m", "e[l] = old[b] + (target - C[b]) / m[b] * width;",
     "e[l] = old[b] + (target - C[b]) * m[b] * width;"),
    # combination
    ("combination weights", "wisum += I[k] / var[k];", "wisum += I[k] / sqrt(var[k]);"),
    ("chi^2 degrees of freedom", "*chi2_dof = K > 1 ? chi2 / (K - 1) : 0.0;",
     "*chi2_dof = K > 1 ? chi2 / K : 0.0;"),
    # integration box
    ("box Jacobian", "                J *= jb->box_w[k];", "                J *= 1.0;"),
    ("box map", "x[k] = jb->box_lo[k] + jb->box_w[k] * x[k];", "x[k] = jb->box_lo[k] + x[k];"),
    # gradient
    ("gradient in mu", "g[1 + k] = fw * 2.0 * u / (a * a);", "g[1 + k] = fw * 2.0 * u / a;"),
    ("gradient in a", "g[dim + 1] = fw * (2.0 * sq / (a * a * a) - dim / a);",
     "g[dim + 1] = fw * (2.0 * sq / (a * a * a) + dim / a);"),
    ("gradient box Jacobian", "                J *= box_w[k];", "                J *= 1.0;"),
    ("gradient variance sums", "s2[c] += (long double)g[c] * g[c];",
     "s2[c] += (long double)g[c];"),
    # more corners
    ("counter without the high word", "ctr[1] = (uint32_t)(i >> 32);", "ctr[1] = 0;"),
    ("Genz discontinuous normalisation", "norm *= (exp(c[k]) - exp(c[k] * a[k])) / c[k];",
     "norm *= (exp(c[k]) - exp(a[k])) / c[k];"),
    ("Genz product-peak normalisation", "atan(c[k] * (1.0 - a[k])) + atan(c[k] * a[k])",
     "atan(c[k] * (1.0 - a[k])) + atan(a[k])"),
    ("mixture without the half", "return 0.5 * (gauss_product(dim, params[0], params + 1, x) +",
     "return 1.0 * (gauss_product(dim, params[0], params + 1, x) +"),
    ("estimate divisor", "*I = S1 / nn;", "*I = S1 / (nn - 1.0);"),
    ("smoothing far end", "out[N - 1] = (hist[N - 2] + hist[N - 1]) / 2.0;",
     "out[N - 1] = (hist[N - 2] + hist[N - 1]) / 3.0;"),
    ("overlapping thread slices",
     "jb->end = first + (uint64_t)(((unsigned __int128)n * (uint64_t)(t + 1)) / (uint64_t)nthreads);",
     "jb->end = first + (uint64_t)(((unsigned __int128)n * (uint64_t)(t + 1)) / (uint64_t)nthreads)"
     " + (t + 1 < nthreads);"),
]


def run_pins(text, workdir, tag):
    """Compile `text` as the oracle and run the pin suite against it: pytest's
    return code (0: every pin passed)."""
    src = os.path.join(workdir, f"{tag}.c")
    lib = os.path.join(workdir, f"lib{tag}.so")
    with open(src, "w") as f:
        f.write(text)
    build_oracle.compile_source(src, lib)
    env = dict(os.environ, VEGAS_ORACLE_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"] + PINS, cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    return r.returncode


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_every_planted_mistake_fails_a_pin(tmp_path):
    original = open(SRC).read()
    for name, old, new in MUTANTS:
        assert original.count(old) == 1, f"{name}: the text to alter must occur once"
    assert run_pins(original, str(tmp_path), "unaltered") == 0, "the harness fails on the oracle"
    with cf.ThreadPoolExecutor(max_workers=4) as ex:
        rcs = list(ex.map(lambda m: run_pins(original.replace(m[1], m[2]), str(tmp_path),
                                             f"mutant{MUTANTS.index(m)}"), MUTANTS))
    survivors = [m[0] for m, rc in zip(MUTANTS, rcs) if rc == 0]
    assert not survivors, f"mistakes no pin caught: {survivors}"
