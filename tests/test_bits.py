"""Integer-arithmetic format conversions of the bucket kernel (csrc/sph_bits.h).

The header is plain C++ with a host/device qualifier.  Here it is compiled
for the host with g++ and checked against the host's IEEE 754 conversions,
which round to nearest with ties to even, as the GPU's cvt.rn does:
float -> double over every one of the 2^32 float bit patterns, double ->
float over random doubles of every exponent with exact ties and the
subnormal, overflow and special cases, and grid index times a power of two
against the FP64 product."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2511_11425_gb300", "csrc")

HARNESS = r"""
#include "sph_bits.h"
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <limits>
using namespace sph::bits;
static uint64_t st = 0x9e3779b97f4a7c15ull;
static uint64_t rnd() {  // SplitMix64
    uint64_t z = (st += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static long bad = 0;
static void chk_d2f(double d) {
    const float a = d2f(d), b = (float)d;
    if (std::isnan(b)) { if (!std::isnan(a)) ++bad; return; }
    if (f_bits(a) != f_bits(b)) {
        if (bad < 5) std::printf("d2f %a: %a vs %a\n", d, (double)a, (double)b);
        ++bad;
    }
}
int main() {
    // float -> double: every bit pattern
    for (uint64_t u = 0; u < (1ull << 32); ++u) {
        const float f = f_from((uint32_t)u);
        const double a = f2d(f), b = (double)f;
        if (std::isnan(b) ? !std::isnan(a) : d_bits(a) != d_bits(b)) {
            if (bad < 5) std::printf("f2d %08x\n", (unsigned)u);
            ++bad;
        }
    }
    // double -> float: random mantissas at every exponent
    for (int E = 0; E < 2048; ++E)
        for (int k = 0; k < 4000; ++k)
            chk_d2f(d_from(((uint64_t)E << 52) | (rnd() & ((1ull << 52) - 1)) |
                           (rnd() & 1 ? 1ull << 63 : 0ull)));
    // exact ties and their neighbours: float-representable values plus half an ulp
    for (int k = 0; k < 2000000; ++k) {
        const uint32_t fb = (uint32_t)rnd() & 0x7f7fffffu;
        const double x = (double)f_from(fb), y = (double)f_from(fb + 1);
        const double mid = 0.5 * (x + y);
        chk_d2f(mid);
        chk_d2f(std::nextafter(mid, 0.0));
        chk_d2f(std::nextafter(mid, 1e300));
        chk_d2f(-mid);
    }
    // boundaries: largest float, overflow threshold, subnormal range
    const double specials[] = {0.0, -0.0, 1.0, -1.0, 3.4028234663852886e38,
                               3.4028235677973366e38, 3.4028235677973362e38, 1e39,
                               std::numeric_limits<double>::infinity(),
                               -std::numeric_limits<double>::infinity(),
                               std::numeric_limits<double>::quiet_NaN(),
                               1.401298464324817e-45, 7.006492321624085e-46,
                               7.006492321624087e-46, 7.006492321624084e-46,
                               2.1019476964872256e-45, 1.1754942106924411e-38,
                               1.1754943508222875e-38, 1.1754942807573643e-38,
                               4.9406564584124654e-324, 2.2250738585072014e-308};
    for (double d : specials) { chk_d2f(d); chk_d2f(-d); }
    for (int sh = 0; sh < 80; ++sh)
        for (int k = 0; k < 20000; ++k)
            chk_d2f(std::ldexp((double)(rnd() >> 11), -1074 + 900 - sh));
    // grid index times a power of two
    for (int k = 0; k < 4000000; ++k) {
        const int v = (int)(uint32_t)rnd() >> (int)(rnd() % 32);
        const double q = std::ldexp(1.0, (int)(rnd() % 120) - 90);
        const double a = i2d_pow2(v, q), b = (double)v * q;
        if (d_bits(a) != d_bits(b)) {
            if (bad < 5) std::printf("i2d %d %a\n", v, q);
            ++bad;
        }
    }
    std::printf("%ld mismatches\n", bad);
    return bad != 0;
}
"""


def test_conversions_match_ieee(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not found")
    src = tmp_path / "bits_check.cpp"
    exe = tmp_path / "bits_check"
    src.write_text(HARNESS)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC, str(src),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout
