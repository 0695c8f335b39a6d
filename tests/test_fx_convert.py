"""Host check of the tile-update epilogue's integer int64 -> FP64 conversion (csrc/fbt_fx.h).

The emulated-FP64 tile product subtracts fx 2^s from C, where fx is the exact 64-bit fixed-point
recombination of the digit-plane group sums.  The FP64-accurate kernel builds the double from
fx's bits with integer instructions; it must equal ldexp((double)fx, s) bit for bit (one rounding
to 53 bits, to nearest with ties to even), so that the kernel's results do not move.  The same
header compiles for the host: this test builds a small C++ driver against it with the system
compiler and compares every case with the C library's conversion, on random magnitudes of 1 to
63 bits, forced ties and near-ties in the dropped bits, both signs, the negation flag, and
exponent shifts that leave the normal range (the ldexp fallback).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2601_11437_gb300", "csrc")

DRIVER = r"""
#include "fbt_fx.h"
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>
static uint64_t bits(double d) { uint64_t b; std::memcpy(&b, &d, 8); return b; }
int main() {
    std::mt19937_64 g(20260101);
    long long bad = 0, n = 0;
    auto check = [&](long long fx, int s, bool neg) {
        const double ref = fx == 0 ? 0.0 : ldexp((double)(neg ? -fx : fx), s);
        const double got = fx_to_double_int(fx, s, neg);
        ++n;
        if (bits(ref) != bits(got)) {
            if (bad < 5) std::printf("mismatch fx=%lld s=%d neg=%d ref=%a got=%a\n", fx, s, (int)neg, ref, got);
            ++bad;
        }
    };
    for (int it = 0; it < 2000000; ++it) {
        const int len = 1 + (int)(g() % 63);
        unsigned long long m = g() & (len == 64 ? ~0ull : ((1ull << len) - 1));
        m |= 1ull << (len - 1);
        const int drop = len - 53;
        if (drop > 0 && g() % 2) {            // the dropped bits exactly half, just below, just above
            const unsigned long long mask = (1ull << drop) - 1, half = 1ull << (drop - 1);
            const int t = (int)(g() % 3);
            m = (m & ~mask) | (t == 0 ? half : (t == 1 ? half - 1 : half + 1));
        }
        const long long fx = (g() & 1) ? -(long long)m : (long long)m;
        const int s = (g() % 4 == 0) ? (int)(g() % 2300) - 1150 : (int)(g() % 200) - 100;
        check(fx, s, (bool)(g() & 1));
    }
    check(0, 5, true);
    check(1, 0, false);
    check(-1, 0, false);
    check(1ll << 62, -1074, true);
    check((((1ll << 53) - 1) << 10) | 0x3FF, 0, false);
    check((((1ll << 53) - 1) << 10) | 0x200, 971, false);
    check(0x7FFFFFFFFFFFFFFFll, 0, false);
    check(-0x7FFFFFFFFFFFFFFFll, -3, true);
    std::printf("%lld cases, %lld mismatches\n", n, bad);
    return bad != 0;
}
"""


def test_integer_conversion_matches_fp64_cast(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "fx_driver.cpp"
    exe = tmp_path / "fx_driver"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "0 mismatches" in out.stdout
