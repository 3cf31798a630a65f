"""Philox4x32-10 outputs from Triton's own implementation, run by Triton's CPU interpreter.

Used as an outside reference for the oracle's Philox (the library routine the generator reduces
to).  Run as a script: reads counters/keys as JSON on stdin, prints outputs as JSON.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox  # noqa: E402


@triton.jit
def _kernel(out_ptr, c0_ptr, c1_ptr, c2_ptr, c3_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    a, b, c, d = philox(seed, tl.load(c0_ptr + i), tl.load(c1_ptr + i), tl.load(c2_ptr + i),
                        tl.load(c3_ptr + i))
    tl.store(out_ptr + 4 * i + 0, a)
    tl.store(out_ptr + 4 * i + 1, b)
    tl.store(out_ptr + 4 * i + 2, c)
    tl.store(out_ptr + 4 * i + 3, d)


def main():
    req = json.load(sys.stdin)
    res = []
    for item in req:
        seed = item["key"][0] | (item["key"][1] << 32)
        ctrs = np.array(item["ctrs"], dtype=np.uint32)       # (N, 4)
        N = ctrs.shape[0]
        cols = [torch.from_numpy(np.ascontiguousarray(ctrs[:, j]).view(np.int32)) for j in range(4)]
        out = torch.zeros(4 * N, dtype=torch.int32)
        _kernel[(1,)](out, *cols, seed, N=N)
        res.append(out.numpy().view(np.uint32).reshape(N, 4).tolist())
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
