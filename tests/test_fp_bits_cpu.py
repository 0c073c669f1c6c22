"""The integer-operation conversions of csrc/fp_bits.cuh (CPU).

The ELBM collision widens FP32 values to FP64 and narrows FP64 values to
FP32 (inputs, seeds, moments, results), and in these helpers does so with integer operations on
the IEEE 754 encodings instead of conversion instructions.  The header
compiles as plain C++, so the same source is built with g++ here and
checked against the C conversions, which follow IEEE 754:
- widen(v) equals (double)v bit for bit for every class of binary32 value:
  zeros, subnormals, normals of every exponent, infinities; NaN stays NaN;
- widen_normal(v) equals (double)v on the normal numbers;
- narrow(x) equals (float)x (round to nearest, ties to even) bit for bit
  for every class of binary64 value, exact ties and subnormal, overflowing
  and underflowing results included; NaN stays NaN;
- narrow_trunc(x) is x truncated toward zero to binary32 (the binary32
  value of largest magnitude not above |x|) on the normal range, zero below
  it and infinity above it;
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1311_2404_gb300", "csrc")

PROGRAM = r"""
#include "fp_bits.cuh"
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <limits>
using namespace lbm;

static uint64_t dbits(double x) { uint64_t b; std::memcpy(&b, &x, 8); return b; }
static uint32_t f32b(float v) { uint32_t b; std::memcpy(&b, &v, 4); return b; }
static double dfrom(uint64_t b) { double x; std::memcpy(&x, &b, 8); return x; }
static float ffrom(uint32_t b) { float v; std::memcpy(&v, &b, 4); return v; }
static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next() {   // splitmix64
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static long fails = 0;
#define CHECK(c, ...) do { if (!(c)) { if (fails < 10) std::printf(__VA_ARGS__); ++fails; } } while (0)

int main() {
    long n_widen = 0, n_trunc = 0;
    // widen: every exponent and sign, fraction patterns (edges and random)
    for (uint32_t s = 0; s < 2; ++s)
        for (uint32_t e = 0; e < 256; ++e)
            for (int k = 0; k < 2000; ++k) {
                uint32_t f = k == 0 ? 0u : k == 1 ? 0x7FFFFFu : k == 2 ? 1u : k == 3 ? 0x400000u
                           : (uint32_t)next() & 0x7FFFFFu;
                const uint32_t b = (s << 31) | (e << 23) | f;
                const float v = ffrom(b);
                const double w = widen(v);
                if (std::isnan(v)) CHECK(std::isnan(w), "widen NaN %08x\n", b);
                else CHECK(dbits(w) == dbits((double)v), "widen %08x\n", b);
                if (e >= 1 && e <= 254)
                    CHECK(dbits(widen_normal(v)) == dbits((double)v), "widen_normal %08x\n", b);
                ++n_widen;
            }
    // narrow and narrow_trunc: binary64 values of every exponent
    for (uint64_t s = 0; s < 2; ++s)
        for (uint64_t e = 0; e < 2048; ++e)
            for (int k = 0; k < 300; ++k) {
                // edges, exact ties at bit 29 and at every subnormal
                // rounding position, one above and below them, random
                const uint64_t tie = 1ull << (28 + (k % 25));
                const uint64_t hi = next() & ~((tie << 1) - 1u) & 0xFFFFFFFFFFFFFull;
                uint64_t f = k == 0 ? 0ull : k == 1 ? 0xFFFFFFFFFFFFFull
                           : k == 2 ? (0x1FFFFFull << 29)
                           : k < 100 ? (hi | tie) + (uint64_t)(k % 3) - 1u
                           : next() & 0xFFFFFFFFFFFFFull;
                f &= 0xFFFFFFFFFFFFFull;
                const double x = dfrom((s << 63) | (e << 52) | f);
                const float rn = narrow(x), cn = (float)x;
                if (std::isnan(x)) CHECK(std::isnan(rn), "narrow NaN %a\n", x);
                else CHECK(f32b(rn) == f32b(cn), "narrow %a: %a vs %a\n", x, (double)rn, (double)cn);
                const float r = narrow_trunc(x);
                const double ax = std::fabs(x);
                if (e < 897) CHECK(r == 0.0f && std::signbit(r) == std::signbit(x), "trunc low %.17g\n", x);
                else if (e > 1150) CHECK(std::isinf(r), "trunc high %.17g\n", x);
                else {
                    const float ar = std::fabs(r);
                    CHECK(std::signbit(r) == std::signbit(x), "trunc sign %.17g\n", x);
                    CHECK((double)ar <= ax, "trunc above %.17g\n", x);
                    const float up = std::nextafter(ar, std::numeric_limits<float>::infinity());
                    CHECK((double)up > ax, "trunc not largest %.17g\n", x);
                }
                ++n_trunc;
            }
    std::printf("widen %ld narrow %ld fails %ld\n", n_widen, n_trunc, fails);
    return fails == 0 ? 0 : 1;
}
"""


def test_fp_bits_against_c_conversions(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "fp_bits_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "fp_bits_check"
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-Wall", "-Wextra", "-Werror", "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
