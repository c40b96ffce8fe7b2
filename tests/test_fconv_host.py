"""The fit's integer-to-binary32 conversions (csrc/ca_fconv.h), compiled for
the host and checked against the C++ compiler's own conversions, which round
to nearest with ties to even: every power of two, the halfway cases around
each rounding point (both tie directions), and a million random values of
every magnitude, for the unsigned 64-bit, signed 64-bit and unsigned 128-bit
forms."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2210_14771_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include <cstdint>
#include <cstring>
#include "ca_fconv.h"

static uint64_t s = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() {   // splitmix64
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static uint32_t bits(float f) { uint32_t b; std::memcpy(&b, &f, 4); return b; }
static long bad = 0, n = 0;
static void u64(uint64_t u) {
    ++n;
    if (bits(ca::u64_to_f32(u)) != bits((float)u)) {
        if (bad++ < 5) std::printf("u64 %llu\n", (unsigned long long)u);
    }
}
static void i64(int64_t v) {
    ++n;
    if (bits(ca::i64_to_f32(v)) != bits((float)v)) {
        if (bad++ < 5) std::printf("i64 %lld\n", (long long)v);
    }
}
static void u128(uint64_t hi, uint64_t lo) {
    ++n;
    const unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
    if (bits(ca::u128_to_f32(hi, lo)) != bits((float)v)) {
        if (bad++ < 5) std::printf("u128 %llx:%llx\n", (unsigned long long)hi, (unsigned long long)lo);
    }
}
int main() {
    u64(0); i64(0); u128(0, 0);
    for (int k = 0; k < 64; ++k) {
        const uint64_t p = 1ull << k;
        for (int64_t d = -3; d <= 3; ++d) { u64(p + d); i64((int64_t)(p + d)); i64(-(int64_t)(p + d)); }
        if (k >= 25) {   // halfway cases: 24 kept bits, then exactly one half
            const uint64_t ulp = 1ull << (k - 23), base = p + 5 * ulp;
            u64(base + ulp / 2); u64(base + ulp + ulp / 2); u64(base + ulp / 2 - 1); u64(base + ulp / 2 + 1);
        }
    }
    i64(INT64_MIN); i64(INT64_MAX); u64(UINT64_MAX);
    for (int k = 0; k < 64; ++k) {
        u128(1ull << k, 0); u128(1ull << k, 1); u128((1ull << k) | 1ull, UINT64_MAX);
        u128(1ull << k, 1ull << 63);
    }
    for (int i = 0; i < 1000000; ++i) {
        const uint64_t r = rnd();
        const int sh = (int)(rnd() % 64);
        u64(r >> sh);
        i64((int64_t)(r >> sh) * ((rnd() & 1) ? -1 : 1));
        u128((r >> sh) >> (rnd() % 2 ? 0 : 30), rnd() >> (rnd() % 64));
    }
    std::printf("checked %ld, mismatches %ld\n", n, bad);
    return bad != 0;
}
"""


def test_integer_to_f32_conversions_round_like_the_compiler(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "fconv.cpp"
    exe = tmp_path / "fconv"
    src.write_text(PROG)
    subprocess.run([gxx, "-O2", "-std=c++17", "-I", HDR, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


RATIO_LIB = r"""
#include <cstdint>
#include "ca_fconv.h"
extern "C" float ratio(int64_t num, int64_t den) { return ca::ratio_to_f32(num, den); }
"""


def test_ratio_rounds_to_the_nearest_binary32(tmp_path):
    """The circumcentre quotient of the fit (csrc/ca_fconv.h, host build):
    the binary32 value nearest to an integer ratio, against exact rational
    rounding on random ratios over the operand range of 4096-pixel frames,
    both signs, and exact halfway cases."""
    import ctypes
    from fractions import Fraction

    import numpy as np
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "ratio.cpp"
    so = tmp_path / "libratio.so"
    src.write_text(RATIO_LIB)
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-I", HDR, str(src), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    lib.ratio.argtypes = [ctypes.c_int64, ctypes.c_int64]
    lib.ratio.restype = ctypes.c_float

    def bits(v):
        return int(np.array(v, np.float32).view(np.uint32))

    def nearest(fr):
        f = np.float32(float(fr))
        best = None
        for c in (np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))):
            d = abs(Fraction(float(c)) - fr)
            if best is None or d < best[0] or (d == best[0] and bits(c) & 1 == 0):
                best = (d, c)
        return best[1]

    rng = np.random.default_rng(5)
    cases = [(1, 3), (-1, 3), (2, 3), (10, -7), ((1 << 37) - 1, 3), (3, (1 << 37) - 1)]
    for _ in range(20000):
        den = int(rng.integers(1, 1 << int(rng.integers(1, 37))))
        num = int(rng.integers(-(1 << int(rng.integers(1, 37))), 1 << 36))
        if num == 0:
            continue
        cases.append((num, den if rng.random() < 0.5 else -den))
    for k in range(3):
        m = (1 << 23) + 999 + k
        cases += [(2 * m + 1, 2), (2 * m + 3, 2), (-(2 * m + 1), -2)]
    for num, den in cases:
        got = lib.ratio(num, den)
        assert bits(got) == bits(nearest(Fraction(num, den))), (num, den, got)
    assert lib.ratio(0, 5) == 0.0
