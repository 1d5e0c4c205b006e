"""Philox4x32-10 computed by Triton's own implementation, run by Triton's CPU
interpreter: a third-party restatement of the same published generator, used
only as a pin for the oracle's Philox.  Usage: python triton_philox_ref.py
ctr.npy key.npy out.npy  (uint32 arrays [n,4], [n,2], [n,4])."""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, k_ptr, out_ptr, n, BLOCK: tl.constexpr):
    i = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=m).to(tl.uint32)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=m).to(tl.uint32)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=m).to(tl.uint32)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=m).to(tl.uint32)
    seed = tl.load(k_ptr + i, mask=m).to(tl.uint64)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a.to(tl.int64), mask=m)
    tl.store(out_ptr + 4 * i + 1, b.to(tl.int64), mask=m)
    tl.store(out_ptr + 4 * i + 2, c.to(tl.int64), mask=m)
    tl.store(out_ptr + 4 * i + 3, d.to(tl.int64), mask=m)


def main():
    ctr = np.load(sys.argv[1]).astype(np.int64)
    key = np.load(sys.argv[2]).astype(np.uint64)
    seed = (key[:, 0] | (key[:, 1] << np.uint64(32))).view(np.int64)
    n = len(ctr)
    out = torch.zeros((n, 4), dtype=torch.int64)
    BLOCK = 64
    _philox_kernel[(triton.cdiv(n, BLOCK),)](torch.from_numpy(ctr.copy()), torch.from_numpy(seed.copy()),
                                             out, n, BLOCK=BLOCK)
    np.save(sys.argv[3], out.numpy().astype(np.uint32))


if __name__ == "__main__":
    main()
