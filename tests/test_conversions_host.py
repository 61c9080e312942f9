"""The integer-only binary32 <-> binary64 conversions of the kernels (f2d, d2f in
rf_device.cuh), compiled as host C++ with the CUDA bit-cast intrinsics written out,
against the host's IEEE 754 conversions (round to nearest even, subnormals kept):
bit for bit over every binary32 exponent, the rounding edges (ties, carries into
the next binade and into infinity, the subnormal and underflow ranges), zeros and
infinities; NaN gives NaN.  Runs without a GPU (g++)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
DEVICE_H = os.path.join(os.path.dirname(HERE), "paper_2202_02319_b300", "csrc", "rf_device.cuh")

HARNESS = r'''
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <random>
#define __device__
#define __noinline__
#define __forceinline__ inline
static inline unsigned __float_as_uint(float f) { unsigned u; std::memcpy(&u, &f, 4); return u; }
static inline float __uint_as_float(unsigned u) { float f; std::memcpy(&f, &u, 4); return f; }
static inline int __double2hiint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(u >> 32); }
static inline int __double2loint(double d) { uint64_t u; std::memcpy(&u, &d, 8); return (int)(uint32_t)u; }
static inline double __hiloint2double(int hi, int lo) {
    uint64_t u = ((uint64_t)(uint32_t)hi << 32) | (uint32_t)lo; double d; std::memcpy(&d, &u, 8); return d;
}
static inline int __clz(unsigned a) { return a ? __builtin_clz(a) : 32; }
static inline unsigned __funnelshift_l(unsigned lo, unsigned hi, unsigned sh) {
    return (unsigned)(((((uint64_t)hi << 32) | lo) << (sh & 31)) >> 32);
}
#include "conversions.inc"
static long bad = 0, n = 0;
static void check_d2f(uint64_t b) {
    double x; std::memcpy(&x, &b, 8);
    const float y = d2f(x), z = (float)x;
    ++n;
    if (std::isnan(x)) { if (!std::isnan(y)) ++bad; return; }
    if (__float_as_uint(y) != __float_as_uint(z)) { if (bad < 5) std::printf("d2f %016llx\n", (unsigned long long)b); ++bad; }
}
static void check_f2d(uint32_t u) {
    const float f = __uint_as_float(u);
    const double y = f2d(f), z = (double)f;
    ++n;
    if (std::isnan(f)) { if (!std::isnan(y)) ++bad; return; }
    if (std::memcmp(&y, &z, 8)) { if (bad < 5) std::printf("f2d %08x\n", u); ++bad; }
}
int main() {
    std::mt19937_64 g(7);
    for (long i = 0; i < 2000000; ++i) check_d2f(g());
    for (long i = 0; i < 2000000; ++i) {
        const uint64_t e = 860 + g() % 300, m = g() & ((1ull << 52) - 1), sg = (g() & 1) << 63;
        const uint64_t b = (e << 52) | m | sg;
        const uint64_t tie = (b & ~0x1FFFFFFFull) | 0x10000000ull;
        check_d2f(b); check_d2f(tie); check_d2f(tie + 1); check_d2f(tie - 1);
    }
    for (long i = 0; i < 500000; ++i) {      // ties on the subnormal grid, exponents 873 .. 896
        const uint64_t e = 873 + g() % 24;
        const unsigned sh = 926 - (unsigned)e;
        const uint64_t M = (1ull << 52) | (g() & ((1ull << 52) - 1));
        const uint64_t tie = (M & ~((1ull << sh) - 1)) | (1ull << (sh - 1));
        for (int d = -1; d <= 1; ++d) check_d2f((e << 52) | ((tie + d) & ((1ull << 52) - 1)));
    }
    for (uint64_t b : {0x0ull, 0x8000000000000000ull, 0x7ff0000000000000ull, 0xfff0000000000000ull,
                       0x47efffffe0000000ull, 0x47efffffefffffffull, 0x47effffff0000000ull, 0x3690000000000000ull,
                       0x36a0000000000000ull, 0x380fffffffffffffull, 0x0000000000000001ull})
        check_d2f(b);
    for (uint64_t u = 0; u < (1ull << 32); u += (u < 0x01000000u || (u > 0x7f000000u && u < 0x81000000u) || u > 0xff000000u) ? 1 : 9973)
        check_f2d((uint32_t)u);
    std::printf("checked %ld mismatches %ld\n", n, bad);
    return bad ? 1 : 0;
}
'''


def _conversion_source():
    text = open(DEVICE_H).read()
    a = text.index("__device__ __noinline__ double f2d_rare")
    b = text.index("// Comparisons of doubles on their bit patterns")
    return text[a:b]


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_conversions_match_host_ieee(tmp_path):
    (tmp_path / "conversions.inc").write_text(_conversion_source())
    (tmp_path / "harness.cpp").write_text(HARNESS)
    exe = tmp_path / "harness"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe), str(tmp_path / "harness.cpp")], check=True,
                   cwd=tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout
