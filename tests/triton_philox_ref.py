"""Philox4x32-10 computed by Triton's own implementation in its CPU interpreter.

Run as a subprocess (TRITON_INTERPRET must be set before triton is imported):
    python triton_philox_ref.py <ctr.npy> <seed> <out.npy>
ctr is uint32[n][4]; out receives uint32[n][4].  Used by the oracle's Philox
pin as an implementation written independently of it.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(seed, cp, op, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(cp + 4 * i + 0)
    c1 = tl.load(cp + 4 * i + 1)
    c2 = tl.load(cp + 4 * i + 2)
    c3 = tl.load(cp + 4 * i + 3)
    a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3, 10)
    tl.store(op + 4 * i + 0, a)
    tl.store(op + 4 * i + 1, b)
    tl.store(op + 4 * i + 2, c)
    tl.store(op + 4 * i + 3, d)


def main():
    ctr = np.load(sys.argv[1]).astype(np.uint32)
    seed = int(sys.argv[2])
    n = ctr.shape[0]
    assert n & (n - 1) == 0, "n must be a power of two"
    c = torch.from_numpy(ctr.reshape(-1).view(np.int32).copy()).view(torch.uint32)
    o = torch.empty_like(c)
    _philox_kernel[(1,)](seed, c, o, N=n)
    np.save(sys.argv[3], o.view(torch.int32).numpy().view(np.uint32).reshape(n, 4))


if __name__ == "__main__":
    main()
