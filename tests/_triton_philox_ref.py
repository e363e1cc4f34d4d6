"""Reference Philox4x32-10 words from Triton's own implementation, run on the
CPU by Triton's interpreter (an independent implementation of the published
generator).  Invoked as a subprocess by test_oracle_philox.py; prints JSON.

usage: python _triton_philox_ref.py <seed> <n> <rng-seed>
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out_ptr, seed, c0_ptr, c1_ptr, c2_ptr, c3_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c0_ptr + i)
    c1 = tl.load(c1_ptr + i)
    c2 = tl.load(c2_ptr + i)
    c3 = tl.load(c3_ptr + i)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)


def main():
    seed, n, rs = int(sys.argv[1]), int(sys.argv[2]), int(sys.argv[3])
    rng = np.random.default_rng(rs)
    ctr = rng.integers(0, 2 ** 32, size=(4, n), dtype=np.uint64)
    ctr[:, 0] = 0                       # include the all-zero counter
    ctr[:, 1] = 0xffffffff              # and the all-ones counter
    cols = [torch.from_numpy(ctr[j].astype(np.uint32).view(np.int32).copy()) for j in range(4)]
    out = torch.zeros(4 * n, dtype=torch.int32)
    _philox_kernel[(1,)](out, seed, *cols, N=n)
    words = (out.numpy().view(np.uint32)).reshape(n, 4)
    print(json.dumps({"ctr": ctr.T.tolist(), "out": words.tolist()}))


if __name__ == "__main__":
    main()
