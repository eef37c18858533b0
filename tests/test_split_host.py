"""The integer split of an FP64 value into float parts (csrc/lp_split.h), which
the gather uses for positions and fields: h = RN(x) and l = RN(x - h) bit for
bit as the host compiler's own conversions give them, over random values,
rounding midpoints, carries into the exponent, both signs and zero; and the
clamped floor the key kernel reads from an FP64 value's bits, against the
library floor.  Compiled with the host C++ compiler; needs no GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2206_11998_gb300", "csrc", "lp_split.h")

PROGRAM = r"""
#include "lp_split.h"
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

static long n = 0, skipped = 0, bad = 0;

static void check(double x)
{
    float h, l;
    if (!lp::split_exact(x, h, l)) { ++skipped; return; }
    const float h0 = (float)x;
    const float l0 = (float)(x - (double)h0);
    uint32_t a, b, c, d;
    memcpy(&a, &h, 4); memcpy(&b, &h0, 4); memcpy(&c, &l, 4); memcpy(&d, &l0, 4);
    ++n;
    if (a != b || c != d) {
        if (bad < 5) printf("mismatch %a: h %a / %a, l %a / %a\n", x, h, h0, l, l0);
        ++bad;
    }
}

int main()
{
    std::mt19937_64 g(7);
    for (long t = 0; t < 3000000; ++t) {
        const uint64_t r = g();
        const int e = (int)(r % 220) - 90;             // inside and outside the handled range
        uint64_t m = g() & 0xfffffffffffffull;
        if (t % 5 == 0) m = (m & ~0x1fffffffull) | 0x10000000ull;   // h's rounding midpoint
        if (t % 11 == 0) m |= 0xfffffe0000000ull;                    // h rounds up into the exponent
        if (t % 13 == 0) m &= ~0x1fffffffull;                        // x is a float: l = 0
        if (t % 17 == 0) m = (m & ~0x1fffffffull) | 0x10000010ull;   // l's own rounding
        const uint64_t b = ((uint64_t)(e + 1023) << 52) | m | ((r >> 63) << 63);
        double x;
        memcpy(&x, &b, 8);
        check(x);
    }
    const double special[] = {0.0, -0.0, 1.0, -1.0, 0.1, -0.1, 1e-22, 5e-23, 3.0e38, 1.7e38,
                              INFINITY, -INFINITY, NAN, 4.9e-324, 2.2250738585072014e-308};
    for (double x : special) check(x);
    // floor_clamped against the library floor on the same kind of values
    long fbad = 0;
    const uint32_t qmax = (1u << 21) - 1u;
    for (long t = 0; t < 2000000; ++t) {
        const uint64_t r = g();
        const int e = (int)(r % 60) - 20;
        uint64_t m = g() & 0xfffffffffffffull;
        if (t % 7 == 0) m = 0;                       // powers of two
        if (t % 9 == 0) m &= ~((1ull << 40) - 1);    // integers and half-integers
        const uint64_t b = ((uint64_t)(e + 1023) << 52) | m | ((t % 10 == 0 ? 1ull : 0ull) << 63);
        double x;
        memcpy(&x, &b, 8);
        const double f = std::floor(x);
        const uint32_t want = !(x >= 0.0) ? 0u : (f >= (double)qmax ? qmax : (uint32_t)f);
        if (lp::floor_clamped(x, qmax) != want) {
            if (fbad < 5) printf("floor mismatch %a: %u / %u\n", x, lp::floor_clamped(x, qmax), want);
            ++fbad;
        }
    }
    const double fs[] = {0.0, -0.0, 0.5, 1.0, 2097151.0, 2097151.5, 2097152.0, 1e300, -1.0, INFINITY, -INFINITY, NAN,
                         4.9e-324};
    const uint32_t fw[] = {0u, 0u, 0u, 1u, qmax, qmax, qmax, qmax, 0u, qmax, 0u, 0u, 0u};
    for (int k = 0; k < 13; ++k)
        if (lp::floor_clamped(fs[k], qmax) != fw[k]) { printf("floor special %a\n", fs[k]); ++fbad; }
    printf("checked %ld skipped %ld bad %ld floor-bad %ld\n", n, skipped, bad, fbad);
    return bad != 0 || fbad != 0 || n < 2000000;
}
"""


def test_split_exact_matches_the_compilers_conversions(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "split_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "split_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    print(r.stdout)
    assert r.returncode == 0, r.stdout
