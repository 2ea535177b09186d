"""The double-float arithmetic of the double-float redo
(csrc/df_arith.cuh), compiled for the host without FMA contraction, against
exact rationals on random normalised pairs: sums within 3 u^2 / (1 - 4 u)
and products within 5 u^2 of the exact results (u = 2^-24), results
normalised (hi = the FP32 rounding of hi + lo), and the sign test v > t and
the order of pairs exact."""
import os
import shutil
import subprocess
from fractions import Fraction as F

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1706_01613_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cstdint>
#include "df_arith.cuh"
using namespace hexval;
static uint64_t st = 88172645463325252ull;
static uint64_t rnd() { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }
static double uni() { return (rnd() >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0; }
static DF pick() {
  double x = uni() * std::ldexp(1.0, (int)(rnd() % 40) - 20);
  float h = (float)x, l = (float)(x - h), s, t;
  fast_two_sum(h, l, s, t);
  return DF(s, t);
}
int main() {
  for (int i = 0; i < 20000; ++i) {
    DF x = pick(), y = pick();
    if (i % 3 == 0) y = DF(-x.hi * (1.0f + std::ldexp((float)uni(), -20)), x.lo * (float)uni());
    DF s = x + y, p = x * y;
    float t = (float)(uni() * std::ldexp(1.0, (int)(rnd() % 40) - 20));
    if (i % 5 == 0) t = x.hi * (1.0f + std::ldexp((float)uni(), -22));
    std::printf("%a %a %a %a %a %a %a %a %a %d %d\n", x.hi, x.lo, y.hi, y.lo, s.hi, s.lo, p.hi,
                p.lo, t, (int)df_gt(x, t), (int)df_less(x, y));
  }
}
"""


@pytest.fixture(scope="module")
def rows(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("df")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return [line.split() for line in out.splitlines()]


def test_sums_products_signs_and_order(rows):
    u2 = F(1, 2 ** 48)
    for w in rows:
        xh, xl, yh, yl, sh, sl, ph, pl, t = [F(float.fromhex(z)) for z in w[:9]]
        gt, less = int(w[9]), int(w[10])
        x, y = xh + xl, yh + yl
        if x + y != 0:
            assert abs(sh + sl - (x + y)) <= 3 * u2 / (1 - 4 * F(1, 2 ** 24)) * abs(x + y)
        else:
            assert sh + sl == 0
        if x * y != 0:
            assert abs(ph + pl - x * y) <= 5 * u2 * abs(x * y)
        for hi, lo in ((sh, sl), (ph, pl)):  # normalised
            assert np.float32(float(hi + lo)) == np.float32(float(hi))
        assert bool(gt) == (x > t)
        assert bool(less) == (x < y or (xh == yh and xl < yl))
        if xh < yh:
            assert x <= y  # the order of normalised pairs
