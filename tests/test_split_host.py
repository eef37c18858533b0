"""The integer split of an FP64 value into float parts (csrc/lp_split.h), which
the gather uses for positions and fields: h = RN(x) and l = RN(x - h) bit for
bit as the host compiler's own conversions give them, over random values,
rounding midpoints, carries into the exponent, both signs and zero.  Compiled
with the host C++ compiler; needs no GPU."""
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
    printf("checked %ld skipped %ld bad %ld\n", n, skipped, bad);
    return bad != 0 || n < 2000000;
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
