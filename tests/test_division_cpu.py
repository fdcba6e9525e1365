"""The quotient the FP64 stage uses: q0 = RN(a y), r = RN(a - b q0) (exact in
an FMA), q = RN(q0 + r y) with y = RN(1/b), which Markstein's theorem makes the
correctly rounded a/b.  A C program (its own restatement of the three steps,
compiled without contraction) compares it with the IEEE quotient on random
operands over a wide exponent range and on significands near all zeros and all
ones, for the constant divisors 6 and 12 and for random divisors."""
import os
import shutil
import subprocess

import pytest

SRC = r"""
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
static uint64_t st = 2210064370ull;
static uint64_t nx(void) { st ^= st << 13; st ^= st >> 7; st ^= st << 17; return st; }
static double pick(int emin, int span, long t) {
  uint64_t b = nx(), e = (uint64_t)(1023 + emin) + (b >> 53) % (uint64_t)span, m = nx() & 0xfffffffffffffull;
  if ((t & 7) == 0) m = (t & 8) ? (0xfffffffffffffull ^ (m & 0xfff)) : (m & 0xfff);
  uint64_t bits = (b & 0x8000000000000000ull) | (e << 52) | m;
  double d; memcpy(&d, &bits, 8); return d;
}
static double quot(double a, double b, double y) {
  double q0 = a * y;
  double r = fma(-q0, b, a);
  return fma(r, y, q0);
}
int main(void) {
  long bad = 0;
  const double cs[2] = {6.0, 12.0};
  for (int k = 0; k < 2; ++k)
    for (long t = 0; t < 4000000; ++t) {
      double a = pick(-900, 1800, t);
      if (quot(a, cs[k], 1.0 / cs[k]) != a / cs[k]) ++bad;
    }
  for (long t = 0; t < 4000000; ++t) {
    double a = pick(-400, 800, t), b = fabs(pick(-300, 600, t >> 3));
    if (quot(a, b, 1.0 / b) != a / b) ++bad;
  }
  printf("%ld\n", bad);
  return 0;
}
"""


def test_markstein_quotient_is_the_ieee_quotient(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "q.c"
    src.write_text(SRC)
    exe = tmp_path / "q"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-o", str(exe), str(src), "-lm"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    assert int(out.strip()) == 0
