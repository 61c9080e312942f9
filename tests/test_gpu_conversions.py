"""The binary32 <-> binary64 conversions the mixed-precision kernels build from
integer operations on the bit fields, against the hardware conversions (round to
nearest even): bit for bit for every non-NaN input, over random bit patterns of
every exponent and the edge cases of the rounding (ties to even, the carry into
the next binade and into infinity, the subnormal and underflow ranges, zeros,
infinities); a NaN input gives a NaN on both sides (the kernels only test for
NaN, so its payload carries nothing)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _bits_equal(a, b):
    """Bit-identical where b is not NaN; NaN exactly where b is NaN."""
    nan = torch.isnan(b)
    if not torch.equal(torch.isnan(a), nan):
        return False
    return bool(torch.equal(a.view(torch.int64)[~nan], b.view(torch.int64)[~nan]))


def _d2f(x64):
    from paper_2202_02319_b300 import native as nv
    xd = torch.as_tensor(x64.view(np.float64)).cuda()
    y, y2 = torch.empty_like(xd), torch.empty_like(xd)
    nv.probe_d2f(xd, y, y2)
    torch.cuda.synchronize()
    return y, y2


def _f2d(u32):
    from paper_2202_02319_b300 import native as nv
    xd = torch.as_tensor(u32.astype(np.uint64).view(np.float64)).cuda()
    y, y2 = torch.empty_like(xd), torch.empty_like(xd)
    nv.probe_f2d(xd, y, y2)
    torch.cuda.synchronize()
    return y, y2


def test_narrowing_matches_hardware_bit_for_bit():
    g = np.random.default_rng(3)
    rand_bits = g.integers(0, 2**63, 4_000_000, dtype=np.int64).astype(np.uint64)
    rand_bits[::2] |= np.uint64(1) << np.uint64(63)                     # both signs
    # doubles whose exponent lies in the binary32 normal range, low 29 bits random
    e = g.integers(897, 1151, 2_000_000, dtype=np.int64).astype(np.uint64)
    mant = g.integers(0, 2**52, 2_000_000, dtype=np.int64).astype(np.uint64)
    normal = (e << np.uint64(52)) | mant
    # exact ties: the 29 dropped bits are 1 followed by zeros, kept mantissa even and odd
    ties = (normal & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    just_above = ties + np.uint64(1)
    just_below = ties - np.uint64(1)
    f32max = float(np.finfo(np.float32).max)
    specials = np.array([
        0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1e-300, -1e-300,
        2.0**-126, np.nextafter(2.0**-126, 0.0), np.nextafter(2.0**-126, 1.0),
        2.0**-149, 2.0**-150, np.nextafter(2.0**-150, 0.0), np.nextafter(2.0**-150, 1.0), 1.5 * 2.0**-150,
        2.0**-140, 3.0 * 2.0**-150, f32max, -f32max, 2.0**128 - 2.0**103, np.nextafter(2.0**128 - 2.0**103, 0.0),
        np.nextafter(2.0**128 - 2.0**103, np.inf), 2.0**128, 1e300, -1e300, np.inf, -np.inf, np.nan,
        1.0, -1.0, np.nextafter(1.0, 2.0), 1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24, 0.1, 300.0, 101325.0,
    ]).view(np.uint64)
    x = np.concatenate([rand_bits, normal, ties, just_above, just_below, specials])
    y, y2 = _d2f(x)
    assert _bits_equal(y, y2)


def test_widening_matches_hardware_bit_for_bit():
    g = np.random.default_rng(4)
    rand = g.integers(0, 2**32, 8_000_000, dtype=np.int64).astype(np.uint32)
    specials = np.array([0.0, -0.0, 1e-45, -1e-45, 1e-40, 1.1754942e-38, 1.17549435e-38, -1.17549435e-38,
                         3.4028235e38, -3.4028235e38, np.inf, -np.inf, np.nan, 1.0, -2.5, 300.0],
                        dtype=np.float32).view(np.uint32)
    edges = np.array([0x00000001, 0x007FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0x7F800001, 0x7FC00000,
                      0x7FFFFFFF, 0x80000000, 0x80800000, 0xFF7FFFFF, 0xFF800000, 0xFFFFFFFF], dtype=np.uint32)
    y, y2 = _f2d(np.concatenate([rand, specials, edges]))
    assert _bits_equal(y, y2)
