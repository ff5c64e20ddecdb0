"""Philox4x32-10 blocks from Triton's own implementation, run by Triton's CPU
interpreter.  Invoked in a subprocess (TRITON_INTERPRET must be set before
Triton is imported).  Reads JSON {"seed": s, "ctr": [[c0,c1,c2,c3], ...]} on
stdin and prints the output blocks as JSON."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(out_ptr, seed, c_ptr, n: tl.constexpr):
    offs = tl.arange(0, n)
    c0 = tl.load(c_ptr + offs * 4 + 0)
    c1 = tl.load(c_ptr + offs * 4 + 1)
    c2 = tl.load(c_ptr + offs * 4 + 2)
    c3 = tl.load(c_ptr + offs * 4 + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, a)
    tl.store(out_ptr + offs * 4 + 1, b)
    tl.store(out_ptr + offs * 4 + 2, c)
    tl.store(out_ptr + offs * 4 + 3, d)


def main():
    req = json.load(sys.stdin)
    ctr = np.array(req["ctr"], dtype=np.int64).reshape(-1)
    n = len(ctr) // 4
    out = torch.zeros(n * 4, dtype=torch.uint32)
    cin = torch.from_numpy(ctr).to(torch.uint32)
    _philox_kernel[(1,)](out, int(req["seed"]), cin, n)
    print(json.dumps(out.to(torch.int64).numpy().reshape(n, 4).tolist()))


if __name__ == "__main__":
    main()
