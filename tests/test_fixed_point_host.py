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
