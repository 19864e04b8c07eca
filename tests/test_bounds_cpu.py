"""Host check of the box-bound comparison the DE repair and the PSO / CSO
clamps use (paper_2505_17430_gb300/csrc/bounds.cuh): the 32-bit integer form
must agree with the IEEE double compares x < b and x > b for every pair --
signed zeros, infinities, NaNs on either side, subnormals, neighbours of the
bounds and random encodings -- since the GPU kernels rely on it to repair
and clamp exactly as the oracle's double compares do."""
import os
import shutil
import subprocess
import tempfile

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_17430_gb300", "csrc")

HARNESS = r"""
#include "bounds.cuh"
#include <float.h>
#include <math.h>
#include <stdio.h>
static double from_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
int main() {
  const double sp[] = {0.0, -0.0, 1.0, -1.0, 100.0, -100.0, INFINITY, -INFINITY, NAN, -NAN,
                       DBL_MIN, -DBL_MIN, DBL_MAX, -DBL_MAX, 4.9e-324, -4.9e-324,
                       nextafter(100.0, 0), nextafter(100.0, 1e9), nextafter(-100.0, 0),
                       nextafter(-100.0, -1e9), 0.5, -0.5,
                       from_bits(0x7FF0000000000001ull), from_bits(0xFFF8000000000000ull),
                       from_bits(0x0000000100000000ull), from_bits(0x00000000FFFFFFFFull),
                       from_bits(0x8000000100000000ull), from_bits(0x80000000FFFFFFFFull)};
  const int ns = (int)(sizeof(sp) / sizeof(sp[0]));
  long bad = 0, n = 0;
  for (int i = 0; i < ns; ++i)
    for (int j = 0; j < ns; ++j) {
      const SvBound b = sv_bound(sp[j]);
      bad += sv_lt_bound(sp[i], b) != (sp[i] < sp[j]);
      bad += sv_gt_bound(sp[i], b) != (sp[i] > sp[j]);
      n += 2;
    }
  uint64_t s = 0x9E3779B97F4A7C15ull;
  for (int t = 0; t < 2000000; ++t) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    const uint64_t s2 = s * 0x2545F4914F6CDD1Dull;
    double x, y;
    if (t % 3 == 0) { x = from_bits(s); y = from_bits(s2); }
    else if (t % 3 == 1) { x = (double)(int64_t)(s >> 11) * 0x1p-44 - 250.0; y = sp[(s2 >> 7) % ns]; }
    else { x = from_bits(s); y = from_bits(s ^ (s2 & 0xFFFFull)); }
    const SvBound b = sv_bound(y);
    bad += sv_lt_bound(x, b) != (x < y);
    bad += sv_gt_bound(x, b) != (x > y);
    n += 2;
  }
  printf("%ld %ld\n", bad, n);
  return 0;
}
"""


def test_bound_compare_matches_ieee():
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        with open(src, "w") as f:
            f.write(HARNESS)
        subprocess.check_call([cxx, "-O2", "-I", CSRC, src, "-o", exe])
        bad, n = map(int, subprocess.check_output([exe]).split())
    assert n > 4_000_000 and bad == 0


U53_HARNESS = r"""
#include "u53.cuh"
#include <stdio.h>
int main() {
  long bad = 0, n = 0;
  uint64_t edge[] = {0ull, 1ull, 2ull, 3ull, (1ull << 52) - 1, 1ull << 52, (1ull << 52) + 1,
                     (1ull << 53) - 1, (1ull << 53) - 2, 1ull << 26, (1ull << 26) - 1};
  for (unsigned i = 0; i < sizeof(edge) / sizeof(edge[0]); ++i, ++n)
    bad += sv_u53_of(edge[i]) != (double)edge[i] * 0x1p-53;
  for (int b = 0; b < 53; ++b, n += 2) {
    bad += sv_u53_of(1ull << b) != (double)(1ull << b) * 0x1p-53;
    bad += sv_u53_of((2ull << b) - 1) != (double)((2ull << b) - 1) * 0x1p-53;
  }
  uint64_t s = 0x243F6A8885A308D3ull;
  for (int t = 0; t < 5000000; ++t, ++n) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    const uint64_t m = (s >> (11 + (t % 40)));  /* every magnitude below 2^53 */
    bad += sv_u53_of(m) != (double)m * 0x1p-53;
  }
  printf("%ld %ld\n", bad, n);
  return 0;
}
"""


def test_u53_integer_construction_matches_conversion():
    """The 53-bit uniform is assembled from integer operations on the GPU
    (u53.cuh, no FP64-pipe conversion); it must be exactly the double of
    m * 2^-53 for every 53-bit m, which the oracle forms by conversion."""
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        with open(src, "w") as f:
            f.write(U53_HARNESS)
        subprocess.check_call([cxx, "-O2", "-I", CSRC, src, "-o", exe])
        bad, n = map(int, subprocess.check_output([exe]).split())
    assert n > 5_000_000 and bad == 0
