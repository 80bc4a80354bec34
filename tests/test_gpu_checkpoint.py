"""Checkpoint / resume: a state exported mid-run and imported into a fresh
workspace continues exactly as the original (samples are functions of their
counters)."""
import numpy as np
import pytest

import paper_2002_12921_b300 as V
from paper_2002_12921_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()


@pytest.mark.parametrize("mode", [V.VEGAS_FP64, V.VEGAS_FP32_EVAL])
def test_resume_equals_uninterrupted_run(mode):
    p = W.gauss_params(5, 0.12, [0.3, 0.45, 0.5, 0.55, 0.7])
    a = V.Vegas(5, 30, 77, mode, W.GAUSS, p, max_iters=8)
    a.config(chunk_samples=70_001)
    a.run([(200_000, 1)] * 3)
    a.iterate(150_000, 1)  # exported between an adapting iteration and its refinement
    blob = a.export_state()
    b = V.Vegas.from_state(blob)
    for v in (a, b):
        v.refine(1.5)
        v.run([(180_000, 1), (300_000, 0)])
    ra, rb = a.iterations(), b.iterations()
    assert ra.shape == rb.shape == (6, 6)
    tol = 1e-12 if mode == V.VEGAS_FP64 else 1e-5
    assert np.allclose(rb[:, 4], ra[:, 4], rtol=tol, atol=0)
    assert np.allclose(b.grid(), a.grid(), rtol=0, atol=1e-14 if mode == V.VEGAS_FP64 else 1e-6)
    assert b.result(4)[3] == 6
    # a blob of the resumed state describes the same run
    assert len(b.export_state()) == len(a.export_state())
    a.close()
    b.close()


def test_import_refuses_a_blob_whose_grid_is_not_increasing():
    """A blob is checked like vegas_set_grid's input: swapping two edges of one
    dimension makes the import fail with VEGAS_EINVAL."""
    import struct

    p = W.gauss_params(3, 0.2)
    a = V.Vegas(3, 10, 5, V.VEGAS_FP64, W.GAUSS, p, max_iters=4)
    a.run([(50_000, 1)] * 2)
    blob = bytearray(a.export_state())
    a.close()
    (nparams,) = struct.unpack_from("<Q", blob, 7 * 8)
    off = 16 * 8 + 8 * nparams + 8 * (11 + 4)  # dimension 1, edges 4 and 5
    e4, e5 = struct.unpack_from("<dd", blob, off)
    struct.pack_into("<dd", blob, off, e5, e4)
    with pytest.raises(V.VegasError) as exc:
        V.Vegas.from_state(bytes(blob))
    assert exc.value.status == V.VEGAS_EINVAL


def test_version_one_blobs_import_and_a_box_needs_version_two():
    """Version 1 had no box: a unit-cube blob relabelled version 1 (word 14 was
    unused and zero) resumes as before; a boxed blob relabelled version 1 has
    2 dim words too many and is refused."""
    import struct

    p = W.gauss_params(3, 0.2)
    for box in (None, [(-1.0, 1.0)] * 3):
        a = V.Vegas(3, 10, 5, V.VEGAS_FP64, W.GAUSS, p, max_iters=4)
        if box:
            a.set_box(box)
        a.run([(50_000, 1)])
        blob = bytearray(a.export_state())
        assert struct.unpack_from("<Q", blob, 8)[0] == 2
        assert struct.unpack_from("<Q", blob, 14 * 8)[0] == (1 if box else 0)
        struct.pack_into("<Q", blob, 8, 1)
        if box is None:
            struct.pack_into("<Q", blob, 14 * 8, 0)
            b = V.Vegas.from_state(bytes(blob))
            assert np.array_equal(b.grid(), a.grid())
            b.close()
        else:
            with pytest.raises(V.VegasError) as exc:
                V.Vegas.from_state(bytes(blob))
            assert exc.value.status == V.VEGAS_EINVAL
        a.close()
