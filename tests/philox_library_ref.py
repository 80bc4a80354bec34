"""Philox4x32-10 words from an independent library implementation.

Runs triton's ``tl.philox`` under triton's CPU interpreter (TRITON_INTERPRET=1),
so it needs no GPU.  Used only as a test pin for the oracle's Philox.  Invoked
as a subprocess: ``python philox_library_ref.py in.npz out.npy`` where in.npz
holds ``ctrs`` (n x 4 uint32) and ``seed`` (uint64; key = (low, high) words).
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(seed_ptr, c_ptr, o_ptr, BLOCK: tl.constexpr):
    offs = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    seed = tl.load(seed_ptr)
    c0 = tl.load(c_ptr + 4 * offs + 0)
    c1 = tl.load(c_ptr + 4 * offs + 1)
    c2 = tl.load(c_ptr + 4 * offs + 2)
    c3 = tl.load(c_ptr + 4 * offs + 3)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(o_ptr + 4 * offs + 0, r0)
    tl.store(o_ptr + 4 * offs + 1, r1)
    tl.store(o_ptr + 4 * offs + 2, r2)
    tl.store(o_ptr + 4 * offs + 3, r3)


def library_philox(ctrs: np.ndarray, seed: int) -> np.ndarray:
    BLOCK = 256
    n = ctrs.shape[0]
    pad = (-n) % BLOCK
    c = np.concatenate([ctrs.astype(np.uint32), np.zeros((pad, 4), np.uint32)])
    ct = torch.from_numpy(c.view(np.int32).copy())
    out = torch.empty_like(ct)
    sd = torch.tensor([np.uint64(seed).astype(np.int64)], dtype=torch.int64)
    _philox_kernel[(c.shape[0] // BLOCK,)](sd, ct, out, BLOCK=BLOCK)
    return out.numpy().view(np.uint32)[:n]


if __name__ == "__main__":
    data = np.load(sys.argv[1])
    res = library_philox(data["ctrs"], int(data["seed"]))
    np.save(sys.argv[2], res)
