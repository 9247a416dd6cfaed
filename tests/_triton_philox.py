"""Evaluate Triton's Philox4x32-10 on the CPU (Triton interpreter) for the oracle pin.

Run as a subprocess: the interpreter switch must be set before Triton loads.
Reads JSON {"ctr": [[4 ints]...], "key": [[2 ints]...]} on stdin and writes the
four output words per counter as JSON on stdout.
"""
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
    c0 = tl.load(c_ptr + 4 * i)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    k0 = tl.load(k_ptr + 2 * i)
    k1 = tl.load(k_ptr + 2 * i + 1)
    o0, o1, o2, o3 = philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(o_ptr + 4 * i, o0)
    tl.store(o_ptr + 4 * i + 1, o1)
    tl.store(o_ptr + 4 * i + 2, o2)
    tl.store(o_ptr + 4 * i + 3, o3)


def main():
    req = json.load(sys.stdin)
    ctr = torch.tensor(req["ctr"], dtype=torch.int64).to(torch.uint32)
    key = torch.tensor(req["key"], dtype=torch.int64).to(torch.uint32)
    n = ctr.shape[0]
    out = torch.empty_like(ctr)
    _kernel[(1,)](ctr, key, out, N=n)
    json.dump([[int(v) & 0xFFFFFFFF for v in row] for row in out.tolist()], sys.stdout)


if __name__ == "__main__":
    main()
