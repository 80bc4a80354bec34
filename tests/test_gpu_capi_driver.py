"""The C ABI from a plain C program (tests/capi_driver.c: cudaMalloc'd
workspace, its own stream, no Python or torch in the process).  Its run of the
Lepage Gaussian equals the Python binding's run on the same seed (FP64 up to
summation order), agrees with the FP64 oracle on the first iteration, and
reaches erf(0.5/a)^d."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import build
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    lib = build.build()
    exe = str(tmp_path_factory.mktemp("capi") / "capi_driver")
    cmd = ["gcc", "-std=c11", "-O2", "-Wall", "-Werror",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA_HOME, "include"),
           os.path.join(ROOT, "tests", "capi_driver.c"),
           "-L", os.path.dirname(lib), "-l:" + os.path.basename(lib),
           "-Wl,-rpath," + os.path.dirname(lib),
           "-L", os.path.join(CUDA_HOME, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(CUDA_HOME, "lib64"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run_driver(exe, mode, seed, dim, nbins, a, n_adapt, k_adapt, n_fixed, k_fixed):
    r = subprocess.run([exe] + [str(x) for x in (mode, seed, dim, nbins, a, n_adapt, k_adapt,
                                                 n_fixed, k_fixed)],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.strip().splitlines()
    I = np.array([float(x) for x in lines[0].split()])
    mean, sigma, chi2, n = lines[1].split()
    return I, float(mean), float(sigma), float(chi2), int(n)


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_c_program_equals_the_binding_and_the_closed_form(driver, mode):
    dim, nbins, a, seed = 4, 50, 0.1, 1
    I, mean, sigma, chi2, n = run_driver(driver, mode, seed, dim, nbins, a, 100_000, 5,
                                         400_000, 2)
    assert n == 7 and I.shape == (7,)
    p = W.gauss_params(dim, a)
    v = V.Vegas(dim, nbins, seed, mode, V.VEGAS_GAUSS, p, max_iters=7)
    v.run([(100_000, 1)] * 5 + [(400_000, 0)] * 2)
    ref = v.iterations()[:, 4]
    v.close()
    # the same counters: summation order alone in FP64; in FP32 a grid that
    # moved by an ulp can round a staged float the other way
    assert np.allclose(I, ref, rtol=1e-13 if mode == V.VEGAS_FP64 else 1e-5, atol=0)
    o = oracle.iterate(oracle.uniform_grid(dim, nbins), seed, 0, 100_000, V.VEGAS_GAUSS, p, True)
    assert abs(I[0] - o["I"]) <= (1e-12 if mode == V.VEGAS_FP64 else 1e-5) * abs(o["I"])
    exact = math.erf(0.5 / a) ** dim
    assert abs(mean - exact) < 5 * sigma and sigma < 1e-3
