"""Philox-4x32-10 words from Triton's own implementation, run on the CPU by
Triton's interpreter (an independent restatement of Salmon et al. 2011 that
the oracle's generator is checked against; test infrastructure only).

Reads {"keys": [[k0, k1], ...], "ctrs": [[c0, c1, c2, c3], ...]} as JSON on
stdin and prints, for every key, the four output words of every counter."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_block(seed_lo, seed_hi, c_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + 4 * i + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + 4 * i + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + 4 * i + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + 4 * i + 3).to(tl.uint32, bitcast=True)
    seed = (seed_hi.to(tl.uint64) << 32) | seed_lo.to(tl.uint64)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, r0.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 1, r1.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 2, r2.to(tl.int32, bitcast=True))
    tl.store(out_ptr + 4 * i + 3, r3.to(tl.int32, bitcast=True))


def main():
    job = json.load(sys.stdin)
    ctrs = job["ctrs"]
    n = len(ctrs)
    assert n & (n - 1) == 0, "counter count must be a power of two"
    flat = [(v & 0xFFFFFFFF) - (1 << 32) if v & 0x80000000 else v for c in ctrs for v in c]
    c = torch.tensor(flat, dtype=torch.int32)
    res = []
    for k0, k1 in job["keys"]:
        out = torch.zeros_like(c)
        _philox_block[(1,)](int(k0), int(k1), c, out, N=n)
        res.append([int(x) & 0xFFFFFFFF for x in out.tolist()])
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
