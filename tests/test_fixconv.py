"""The integer rounding of the DF / DF-P epilogue (fixconv.cuh) against the C
library's IEEE 754 conversion on the host: double -> int64 with llrint in the
default round-to-nearest-even mode, over every exponent the epilogue can
produce, exact halves of either parity and their neighbours, and the range
ends.  The same header compiles into the CUDA kernels; the GPU tests compare
sweeps that use it with sweeps that use the hardware conversion, bit for
bit."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include "fixconv.cuh"

static uint64_t st = 0x9E3779B97F4A7C15ull;
static uint64_t next() {   // SplitMix64
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double from_bits(uint64_t b) { double x; std::memcpy(&x, &b, sizeof x); return x; }
static long bad = 0, checked = 0;
static void check(double y) {
  long long want = llrint(y);
  long long got = fixconv::f64_to_i64_rn(y);
  checked++;
  if (want != got && bad++ < 10) printf("f64_to_i64_rn(%a): %lld != %lld\n", y, got, want);
}
int main() {
  check(0.0);
  check(0.5);
  check(1.5);
  check(2.5);
  check(4.9406564584124654e-324);
  check(0.49999999999999994);
  check(std::nextafter(0.5, 1.0));
  for (int e = -40; e < 63; e++)
    for (int i = 0; i < 20000; i++) check(from_bits(((uint64_t)(1023 + e) << 52) | (next() & ((1ull << 52) - 1))));
  for (int i = 0; i < 200000; i++) {
    const uint64_t nn = next() >> (12 + next() % 52);   // n + 0.5 is exact for n < 2^52
    check((double)nn + 0.5);
    check((double)nn);
    check(std::nextafter((double)nn + 0.5, 0.0));
    check(std::nextafter((double)nn + 0.5, 1e300));
  }
  check(std::nextafter(9223372036854775808.0, 0.0));
  printf("checked %ld, mismatches %ld\n", checked, bad);
  return bad != 0;
}
"""


def test_fixconv_matches_ieee_rounding(tmp_path):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not found")
    src = tmp_path / "fixconv_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "fixconv_check"
    inc = os.path.join(ROOT, "paper_2401_15870_gb300", "csrc")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", inc, str(src), "-o", str(exe)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
