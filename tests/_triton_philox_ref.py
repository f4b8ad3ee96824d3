"""Independent Philox4x32-10 reference: Triton's own implementation run by
Triton's CPU interpreter.  Usage: python _triton_philox_ref.py SEED C0 C1 C2 C3 N
prints N lines of four uint32 words for counters (C0+i, C1, C2, C3)."""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _k(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a, mask=m)
    tl.store(out_ptr + 4 * i + 1, b, mask=m)
    tl.store(out_ptr + 4 * i + 2, c, mask=m)
    tl.store(out_ptr + 4 * i + 3, d, mask=m)


def main():
    seed, c0, c1, c2, c3, n = (int(v) for v in sys.argv[1:7])
    ctr = np.zeros((n, 4), dtype=np.uint32)
    ctr[:, 0] = (c0 + np.arange(n)).astype(np.uint32)
    ctr[:, 1], ctr[:, 2], ctr[:, 3] = c1, c2, c3
    out = torch.zeros(n, 4, dtype=torch.int32)
    block = 1 << max(0, (n - 1).bit_length())
    _k[(1,)](out, torch.from_numpy(ctr.view(np.int32)), seed, n, BLOCK=block)
    for row in out.numpy().view(np.uint32):
        print(*row)


if __name__ == "__main__":
    main()
