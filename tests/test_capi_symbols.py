"""The C-ABI library loads and exports every symbol include/vegas.h declares
(CPU only: no call here reaches the GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vegas.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(vegas_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return V.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(V.binding.EXPORTED)


def test_workspace_bytes_validation(lib):
    b = V.vegas_workspace_bytes(8, 50, 64)
    assert b % 256 == 0 and b >= 8 * 51 * 8 + 8 * 50 * 8 + 64 * 8 * 8
    assert V.vegas_workspace_bytes(16, 512, 1) > V.vegas_workspace_bytes(16, 100, 1)
    for args in [(0, 50, 1), (21, 50, 1), (8, 0, 1), (8, 1025, 1), (16, 600, 1), (8, 50, 0)]:
        with pytest.raises(V.VegasError) as e:
            V.vegas_workspace_bytes(*args)
        assert e.value.status == V.VEGAS_EINVAL


def test_init_rejects_bad_arguments_before_touching_a_device(lib):
    h = ctypes.c_void_p()
    p = (ctypes.c_double * 5)(0.1, 0.5, 0.5, 0.5, 0.5)
    ws = V.vegas_workspace_bytes(4, 50, 8)
    # no workspace
    assert lib.vegas_init_grid(ctypes.byref(h), 4, 50, 1, 0, 0, p, 5, 8, None, ws, None) == 1
    # misaligned workspace pointer
    assert lib.vegas_init_grid(ctypes.byref(h), 4, 50, 1, 0, 0, p, 5, 8, 0x1008, ws, None) == 1
    # too small
    assert lib.vegas_init_grid(ctypes.byref(h), 4, 50, 1, 0, 0, p, 5, 8, 0x10000, ws - 256,
                               None) == V.VEGAS_ENOSPACE
    # bad mode, bad shape
    assert lib.vegas_init_grid(ctypes.byref(h), 4, 50, 1, 7, 0, p, 5, 8, 0x10000, ws, None) == 1
    assert lib.vegas_init_grid(ctypes.byref(h), 40, 50, 1, 0, 0, p, 5, 8, 0x10000, ws, None) == 1
    assert h.value is None
    assert lib.vegas_destroy(None) == 0
    assert lib.vegas_iterate(None, 100, 1) == 1
    assert lib.vegas_sample_words(1, 0, 0, 0, 10, 0, None, None) == 1


def test_strerror_covers_codes(lib):
    texts = {V.vegas_strerror(c) for c in range(6)}
    assert len(texts) == 6 and V.vegas_strerror(99) == "unknown status"


def test_import_rejects_malformed_blobs_without_a_device(lib):
    h = ctypes.c_void_p()
    bad = b"NOTVEGAS" + bytes(200)
    assert lib.vegas_import_state(ctypes.byref(h), bad, len(bad), None, 0, None) == 1
    short = b"VEGASB3\x00" + bytes(16)
    assert lib.vegas_import_state(ctypes.byref(h), short, len(short), None, 0, None) == 1
    assert h.value is None


def test_user_integrand_descriptors_load_without_a_device(lib):
    """A caller's integrand file compiles against include/vegas_user_integrand.cuh
    and its descriptors carry the compiled dimension and callbacks; the
    library rejects one without a state."""
    so = build.build_user_integrand(os.path.join(ROOT, "tests", "user_integrands.cu"),
                                    os.path.join(ROOT, "tests", "_build", "libuser_integrands.so"))
    sizes = set()
    for name, dim in [("user_gauss_d4", 4), ("user_gauss_d8", 8), ("user_sum_square_d5", 5),
                      ("user_sine_d3", 3)]:
        mod, addr = V.load_user_integrand(so, name)
        desc = V.vegas_user_integrand.from_address(addr)
        assert desc.dim == dim and desc.prepare and desc.launch
        sizes.add(desc.args_bytes)
    assert len(sizes) == 1 and sizes.pop() > 0
    assert lib.vegas_set_user_integrand(None, addr, None) == V.VEGAS_EINVAL


def test_fp64_exp_table_is_correctly_rounded_powers_of_two():
    """The 256-entry table of the FP64 path's exponential holds 2^(j/256)
    rounded to the nearest double (checked against 200-bit arithmetic)."""
    import mpmath

    mpmath.mp.prec = 200
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2002_12921_b300", "csrc", "exp2_table.h")
    vals = [float.fromhex(h) for h in re.findall(r"0x[0-9a-f.]+p[+-]\d+", open(path).read())]
    assert len(vals) == 256
    for j, v in enumerate(vals):
        exact = mpmath.mpf(2) ** (mpmath.mpf(j) / 256)
        assert abs(mpmath.mpf(v) - exact) <= mpmath.mpf(np.spacing(v)) / 2, j


def test_sample_words_refuses_counts_beyond_the_index_bound(lib):
    """vegas_sample_words checks n against VEGAS_MAX_SAMPLE_INDEX before any
    device work (the pointer is never touched)."""
    import ctypes

    rc = lib.vegas_sample_words(1, 0, 0, 0, V.binding.VEGAS_MAX_SAMPLE_INDEX + 1, 4,
                                ctypes.c_void_p(0x1000), None)
    assert rc == V.VEGAS_EINVAL


def test_binding_constants_equal_the_header():
    """The binding's copies of the header's limits and status codes are the
    values include/vegas.h defines."""
    import os
    import re

    header = open(os.path.join(os.path.dirname(__file__), "..", "include", "vegas.h")).read()
    defines = {m.group(1): int(m.group(2).rstrip("uUlL"), 0)
               for m in re.finditer(r"^#define\s+(VEGAS_\w+)\s+(0x[0-9A-Fa-f]+\w*|-?\d+)\b",
                                    header, re.M)}
    names = ["VEGAS_MAX_DIM", "VEGAS_MAX_BINS", "VEGAS_MAX_DIM_X_BINS", "VEGAS_MAX_DEVICES",
             "VEGAS_MAX_SAMPLE_INDEX", "VEGAS_OK", "VEGAS_EINVAL", "VEGAS_ECUDA",
             "VEGAS_ENONFINITE", "VEGAS_ESTATE", "VEGAS_ENOSPACE", "VEGAS_FP64",
             "VEGAS_FP32_EVAL", "VEGAS_GAUSS", "VEGAS_GAUSS_MIX2", "VEGAS_FLAT",
             "VEGAS_GENZ_DISC", "VEGAS_GENZ_PPEAK", "VEGAS_USER"]
    for n in names:
        assert n in defines, n
        assert getattr(V.binding, n) == defines[n], n
