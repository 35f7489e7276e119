"""Independent Philox4x32-10 outputs from triton's implementation, run in triton's CPU
interpreter. Invoked as a subprocess by the oracle pin (the interpreter must be chosen
before triton is imported). Reads counters/keys as JSON on stdin, writes outputs."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402
from triton.language.random import philox_impl  # noqa: E402


@triton.jit
def _kernel(c_ptr, k_ptr, o_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    k0 = tl.load(k_ptr + 2 * i + 0)
    k1 = tl.load(k_ptr + 2 * i + 1)
    o0, o1, o2, o3 = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(o_ptr + 4 * i + 0, o0)
    tl.store(o_ptr + 4 * i + 1, o1)
    tl.store(o_ptr + 4 * i + 2, o2)
    tl.store(o_ptr + 4 * i + 3, o3)


def main():
    req = json.load(sys.stdin)
    ctrs, keys = req["ctr"], req["key"]
    n = len(ctrs)
    N = 1
    while N < n:
        N *= 2
    c = torch.zeros(4 * N, dtype=torch.int64)
    k = torch.zeros(2 * N, dtype=torch.int64)
    for i in range(n):
        for j in range(4):
            c[4 * i + j] = ctrs[i][j]
        for j in range(2):
            k[2 * i + j] = keys[i][j]
    c32 = c.to(torch.uint32)
    k32 = k.to(torch.uint32)
    o = torch.zeros(4 * N, dtype=torch.uint32)
    _kernel[(1,)](c32, k32, o, N)
    out = [[int(x) & 0xFFFFFFFF for x in o[4 * i:4 * i + 4].to(torch.int64)] for i in range(n)]
    json.dump(out, sys.stdout)


if __name__ == "__main__":
    main()
