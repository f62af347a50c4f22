"""Evaluate Philox4x32-10 with the triton library's implementation on the CPU.

Run as a subprocess (the interpreter switch must be set before triton is
imported).  Reads counters and keys as JSON from argv[1], prints outputs as JSON.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _philox_kernel(out, cp, kp, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    c0 = tl.load(cp + 4 * i).to(tl.uint32, bitcast=True)
    c1 = tl.load(cp + 4 * i + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(cp + 4 * i + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(cp + 4 * i + 3).to(tl.uint32, bitcast=True)
    k0 = tl.load(kp + 2 * i).to(tl.uint32, bitcast=True)
    k1 = tl.load(kp + 2 * i + 1).to(tl.uint32, bitcast=True)
    a, b, c, d = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out + 4 * i, a.to(tl.int32, bitcast=True))
    tl.store(out + 4 * i + 1, b.to(tl.int32, bitcast=True))
    tl.store(out + 4 * i + 2, c.to(tl.int32, bitcast=True))
    tl.store(out + 4 * i + 3, d.to(tl.int32, bitcast=True))


def main():
    spec = json.loads(sys.argv[1])
    ctr = np.array(spec["ctr"], dtype=np.uint32).reshape(-1, 4)
    key = np.array(spec["key"], dtype=np.uint32).reshape(-1, 2)
    n = ctr.shape[0]
    block = 1
    while block < n:
        block *= 2
    ctr = np.concatenate([ctr, np.zeros((block - n, 4), np.uint32)])
    key = np.concatenate([key, np.zeros((block - n, 2), np.uint32)])
    out = torch.zeros(4 * block, dtype=torch.int32)
    _philox_kernel[(1,)](out, torch.from_numpy(ctr.view(np.int32).ravel().copy()),
                         torch.from_numpy(key.view(np.int32).ravel().copy()), BLOCK=block)
    res = out.numpy().view(np.uint32).reshape(block, 4)[:n]
    print(json.dumps(res.astype(np.int64).tolist()))


if __name__ == "__main__":
    main()
