"""Philox4x32-10 computed by triton's own ``tl.philox`` in triton's CPU interpreter.

Run as a script (``TRITON_INTERPRET=1`` must be set before triton is imported,
so tests call it in a subprocess).  Reads a .npz with ``ctr`` (k x 4 uint32)
and ``seeds`` (s uint64) and writes ``out`` (s x k x 4 uint32).  This is an
independent library implementation used only to pin the oracle's Philox.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(ctr_ptr, out_ptr, seed, K: tl.constexpr):
    i = tl.arange(0, K)
    c0 = tl.load(ctr_ptr + 4 * i + 0)
    c1 = tl.load(ctr_ptr + 4 * i + 1)
    c2 = tl.load(ctr_ptr + 4 * i + 2)
    c3 = tl.load(ctr_ptr + 4 * i + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)


def main(inp, outp):
    z = np.load(inp)
    ctr = z["ctr"].astype(np.uint32)
    k = ctr.shape[0]
    assert k & (k - 1) == 0, "row count must be a power of two"
    ctr_t = torch.from_numpy(ctr.view(np.int32).copy())
    res = []
    for s in z["seeds"].astype(np.uint64).tolist():
        out = torch.zeros(k * 4, dtype=torch.int32)
        # tl.philox splits the 64-bit seed into (lo32, hi32) as the Philox key
        _philox_kernel[(1,)](ctr_t, out, int(s) if s < (1 << 63) else int(s) - (1 << 64), K=k)
        res.append(out.numpy().view(np.uint32).reshape(k, 4))
    np.savez(outp, out=np.stack(res))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
