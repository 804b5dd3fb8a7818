"""Philox4x32-10 reference values from Triton's own implementation.

Run under ``TRITON_INTERPRET=1`` (Triton's CPU interpreter).  Reads a JSON
list of ``[counter(4 words), key(2 words)]`` on stdin and prints the four
output words of each.  Triton's ``tl.philox(seed, c0, c1, c2, c3)`` uses the
64-bit seed as the key (low word, high word), which is the keying the oracle
documents; it is an implementation written independently of this project.
"""
import json
import os
import sys

assert os.environ.get("TRITON_INTERPRET") == "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(ctr_ptr, out_ptr, seed):
    c0 = tl.load(ctr_ptr + 0)
    c1 = tl.load(ctr_ptr + 1)
    c2 = tl.load(ctr_ptr + 2)
    c3 = tl.load(ctr_ptr + 3)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 0, a)
    tl.store(out_ptr + 1, b)
    tl.store(out_ptr + 2, c)
    tl.store(out_ptr + 3, d)


def main():
    cases = json.loads(sys.stdin.read())
    res = []
    for ctr, key in cases:
        seed = int(key[0]) | (int(key[1]) << 32)
        if seed >= 2**63:
            seed -= 2**64
        c = torch.tensor(np.array(ctr, dtype=np.uint32).view(np.int32))
        out = torch.zeros(4, dtype=torch.int32)
        _kernel[(1,)](c, out, seed)
        res.append([int(v) & 0xFFFFFFFF for v in out.tolist()])
    print(json.dumps(res))


if __name__ == "__main__":
    main()
