"""Host checks of the fixed-point arithmetic of the 3-D FP64 residual kernel (k_resid3d_fx):
the two conversion helpers are taken verbatim from csrc/kernels.cuh, compiled for the host
with g++ behind small shims for the CUDA bit-cast intrinsics, and compared on random inputs
with exact references (x 2^S rounded to the nearest integer through long double; int64 to
double through the compiler's correctly rounded conversion).  The overflow-safety bound of
the exact stencil sum T = 16 s1 - s2 - 90 x is checked against the ghost-cell formulas of
Eqs. (velBCHomoDiri5th) and (Neumann5) as the oracle states them."""
import os
import re
import shutil
import subprocess

import pytest

from oracle import stencil

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNELS = os.path.join(ROOT, "paper_2506_02663_gb300", "csrc", "kernels.cuh")

SHIMS = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#define __device__
#define __forceinline__ inline
static long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static double __longlong_as_double(long long b) { double x; std::memcpy(&x, &b, 8); return x; }
static int __clzll(long long v) { return v == 0 ? 64 : __builtin_clzll((unsigned long long)v); }
static unsigned __funnelshift_r(unsigned lo, unsigned hi, unsigned s) {
  return (unsigned)((((unsigned long long)hi << 32) | lo) >> (s & 31));
}
"""

MAIN = r"""
int main() {
  std::mt19937_64 g(20250603);
  long bad = 0;
  for (int it = 0; it < 2000000; ++it) {            // int64 -> FP64, round to nearest even
    long long t = (long long)g() >> (g() % 64);
    if (fx_to_double(t) != (double)t) ++bad;
  }
  for (long long base : {(1LL << 53) + 1, (1LL << 54) + 2, (1LL << 60) + (1LL << 7), (1LL << 60) + 3 * (1LL << 7)})
    for (long long s : {1LL, -1LL})
      if (fx_to_double(s * base) != (double)(s * base)) ++bad;   // ties
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  for (int it = 0; it < 1000000; ++it) {            // FP64 -> frame, ties away from zero
    const double mx = std::fabs(std::ldexp(1.0, (int)(g() % 200) - 100) * (0.5 + 0.5 * U(g) * U(g)));
    long long mb; std::memcpy(&mb, &mx, 8);
    const int emax = (int)((mb >> 52) & 0x7ff);
    const double x = mx * U(g) * std::ldexp(1.0, -(int)(g() % 60));
    bool ovf = false;
    const long long v = fx_of(x, emax, 2, ovf);
    const long double r = std::round(std::ldexp((long double)x, 1075 - emax));
    if (ovf || (long double)v != r) ++bad;
    bool o = false;
    if (fx_of(mx, emax, 2, o) >= (1LL << 53) || o) ++bad;                 // the maximum maps below 2^53
    const double y = mx * (1.0 + 2.9 * std::fabs(U(g))) * (U(g) < 0.0 ? -1.0 : 1.0);  // inside the headroom
    bool oy = false;
    const long long vy = fx_of(y, emax, 2, oy);
    if (oy || (long double)vy != std::round(std::ldexp((long double)y, 1075 - emax))) ++bad;
    const double lim2 = std::ldexp(1.0, emax - 1020), lim7 = std::ldexp(1.0, emax - 1015);
    bool a = false, b = false, c = false, d = false;
    fx_of(std::nextafter(lim2, 0.0), emax, 2, a);
    fx_of(lim2, emax, 2, b);
    fx_of(std::nextafter(lim7, 0.0), emax, 7, c);
    fx_of(lim7, emax, 7, d);
    if (a || !b || c || !d) ++bad;                                        // headroom 2^2 and 2^7
    bool e = false;
    if (fx_of(0.0, emax, 2, e) != 0 || e) ++bad;
    bool f = false;
    fx_of(INFINITY, emax, 7, f);
    if (!f) ++bad;
  }
  std::printf("bad = %ld\n", bad);
  return bad != 0;
}
"""


def _extract(src, signature):
    i = src.index(signature)
    j = src.index("\n}\n", i)
    return src[i:j + 3]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_fixed_point_conversions_are_exact(tmp_path):
    src = open(KERNELS).read()
    body = (_extract(src, "__device__ __forceinline__ long long fx_of(") +
            _extract(src, "__device__ __forceinline__ double fx_to_double("))
    cpp = tmp_path / "fx.cpp"
    cpp.write_text(SHIMS + body + MAIN)
    exe = tmp_path / "fx"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe), str(cpp)], check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "bad = 0" in r.stdout, r.stdout + r.stderr


def test_fixed_point_sum_cannot_overflow():
    """|T| / 2^53 for the worst cell (one ghost per direction, layer 1 in s1 and layer 2 in s2,
    stored ghosts below 4, interior values below 1) stays below 2^10, so T fits in int64."""
    c = {layer: max(sum(abs(float(v)) for v in tab[layer][0]) for tab in (stencil.DIRICHLET, stencil.NEUMANN))
         for layer in (1, 2)}
    assert abs(c[2] - 1012 / 12) < 1e-12  # Dirichlet layer 2 is the largest
    g1, g2 = max(c[1], 4.0), max(c[2], 4.0)
    worst = 16 * (3 * g1 + 3) + (3 * g2 + 3) + 90
    assert worst < 1024, worst
    # the kernel's comment states the same bound
    assert re.search(r"\(16 \(3 \* 11\.7 \+ 3\) \+ 3 \* 84\.4 \+ 3 \+ 90\) 2\^53 < 2\^63", open(KERNELS).read())


CONV_SHIMS = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#define __device__
#define __forceinline__ inline
static long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static unsigned __float_as_uint(float x) { unsigned b; std::memcpy(&b, &x, 4); return b; }
static float __uint_as_float(unsigned b) { float x; std::memcpy(&x, &b, 4); return x; }
static double __hiloint2double(int hi, int lo) {
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
  double x; std::memcpy(&x, &b, 8); return x;
}
"""

CONV_MAIN = r"""
static bool same64(double a, double b) { return std::memcmp(&a, &b, 8) == 0; }
static bool same32(float a, float b) { return std::memcmp(&a, &b, 4) == 0; }
int main() {
  std::mt19937_64 g(20250604);
  long bad = 0;
  // FP32 -> FP64: random bit patterns (every class), and the special values
  for (int it = 0; it < 4000000; ++it) {
    const float f = __uint_as_float((unsigned)g());
    if (std::isnan(f)) continue;
    if (!same64(f32_to_f64(f), (double)f)) ++bad;
  }
  for (float f : {0.0f, -0.0f, 1.0f, -1.0f, INFINITY, -INFINITY, 1.17549435e-38f, 1.4e-45f, 3.4028235e38f})
    if (!same64(f32_to_f64(f), (double)f)) ++bad;
  // FP64 -> FP32: random doubles over the FP32 range and beyond, exact ties, the range ends
  std::uniform_int_distribution<int> ex(860, 1180);
  for (int it = 0; it < 4000000; ++it) {
    unsigned long long b = g();
    b = (b & 0x800fffffffffffffull) | ((unsigned long long)ex(g) << 52);
    if (it % 4 == 1) b = (b & ~0x1fffffffull) | 0x10000000ull;                 // a tie
    if (it % 4 == 2) b = (b & ~0x1fffffffull) | (g() & 1 ? 0x0fffffffull : 0x10000001ull);
    double d; std::memcpy(&d, &b, 8);
    if (!same32(f64_to_f32(d), (float)d)) ++bad;
  }
  for (double d : {0.0, -0.0, 1.0, -1.0, (double)INFINITY, -(double)INFINITY, 3.4028235677973366e38, 3.4028235e38 * 1.0000001,
                   1.1754943508222875e-38, 1.1754942e-38, 1e-45, 1e300, -1e-300})
    if (!same32(f64_to_f32(d), (float)d)) ++bad;
  std::printf("bad = %ld\n", bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_precision_conversions_match_the_casts(tmp_path):
    """The integer-instruction FP32 <-> FP64 conversions of the refinement loop (taken
    verbatim from csrc/kernels.cuh) against the compiler's casts, bit for bit: FP32 -> FP64
    on random bit patterns of every class; FP64 -> FP32 (round to nearest even) on random
    doubles from below the smallest normal float to above the largest, exact ties, and the
    ends of the range (overflow to infinity, subnormal results)."""
    src = open(KERNELS).read()
    body = (_extract(src, "__device__ __forceinline__ double f32_to_f64(") +
            _extract(src, "__device__ __forceinline__ float f64_to_f32("))
    cpp = tmp_path / "conv.cpp"
    cpp.write_text(CONV_SHIMS + body + CONV_MAIN)
    exe = tmp_path / "conv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(cpp)], check=True,
                   capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "bad = 0" in r.stdout, r.stdout + r.stderr
