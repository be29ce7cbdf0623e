"""CPU check of the host side of the GPU quantizer (Sec. III-B).

The kernels quantize with constants the host derives per attribute
(jiffy::make_attr in csrc/jiffy_types.h): a 32-bit multiplier and shift on
the input clamped at `lim`, or a 64-bit reciprocal when no 32-bit multiplier
divides every 32-bit dividend exactly. This test compiles that header with the
host compiler, evaluates the kernel's arithmetic with those constants on edge
and random samples, and compares every result with the oracle's quantizer.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2209_08196_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "jiffy_types.h"
// reads lines "s P v", prints the kernel-side q
int main() {
  unsigned s, P, v;
  while (std::scanf("%u %u %u", &s, &P, &v) == 3) {
    const jiffy::AttrDev a = jiffy::make_attr(s, P);
    uint32_t q;
    if (a.qkind == 0) {
      q = v;
    } else if (a.qkind == 1) {
      const uint32_t n = (v < a.lim ? v : a.lim) + a.half;
      q = (uint32_t)(((uint64_t)n * a.m32) >> 32) >> a.sh;
    } else {  // 64-bit reciprocal path
      const unsigned long long n = (unsigned long long)v + (a.P >> 1);
      if (a.P <= 0x80000000u) q = (uint32_t)(((unsigned __int128)n * a.magic) >> 64);
      else q = (uint32_t)(n >= a.P) + (uint32_t)(n >= 2ull * a.P);
      q = q < a.qmax ? q : a.qmax;
    }
    std::printf("%u %u\n", a.qkind, q);
  }
  return 0;
}
"""


def _cases():
    rng = np.random.default_rng(7)
    out = []
    precisions = [1, 2, 3, 5, 7, 10, 11, 100, 641, 1000, 4095, 65535, 65536, 65537, 6700417,
                  (1 << 30) - 1, 1 << 30, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFE, 0xFFFFFFFF]
    precisions += [int(x) for x in rng.integers(2, 100000, 40)] + [int(x) for x in rng.integers(2, 1 << 32, 20)]
    for s in (1, 2, 4):
        mx = (1 << (8 * s)) - 1
        for P in precisions:
            vals = {0, 1, mx, mx - 1, P // 2, P - 1, P, P + P // 2, min(mx, P * 3 + P // 2)}
            q = mx // P
            for k in (q - 1, q, q + 1):
                for d in (-1, 0, 1):
                    v = k * P + P // 2 + d
                    if 0 <= v <= mx:
                        vals.add(v)
            vals |= {int(x) for x in rng.integers(0, mx + 1, 25, dtype=np.uint64)}
            out += [(s, P, v) for v in sorted(vals)]
    return out


@pytest.mark.skipif(shutil.which("g++") is None, reason="no host C++ compiler")
def test_kernel_quantizer_constants_match_the_oracle():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "q.cpp")
        exe = os.path.join(d, "q")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.check_call(["g++", "-O1", "-std=c++17", "-I" + CSRC, src, "-o", exe])
        cases = _cases()
        inp = "".join("%d %d %d\n" % c for c in cases)
        res = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    kinds = set()
    for (s, P, v), line in zip(cases, res):
        kind, q = (int(x) for x in line.split())
        kinds.add(kind)
        assert q == oracle.quantize(v, P, s), (s, P, v, kind)
    assert kinds == {0, 1, 2}  # every kernel path was exercised
