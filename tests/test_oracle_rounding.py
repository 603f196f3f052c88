"""Pins for the storage rounding of the oracle's precision form (FP32 and
BF16 history entries) against literal bit patterns: round to nearest with
ties to even, the overflow threshold, NaN, signed zero and subnormals.  The
BF16 entries are rounded through FP32 (FP64 -> FP32 to nearest, then
FP32 -> BF16 to nearest even), the same two steps the device takes; the
double-rounding case at the end pins that choice.

BF16 keeps the top 16 bits of an IEEE binary32: 1 sign, 8 exponent and 7
fraction bits, so the spacing just above 1.0 is 2^-7."""
import math
import struct

import pytest


def bits32(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def from_bits32(b: int) -> float:
    return struct.unpack("<f", struct.pack("<I", b))[0]


BF16_CASES = [
    # (input, expected BF16 bit pattern (the top 16 bits of the float))
    (1.0, 0x3F80),
    (1.0 + 2.0 ** -7, 0x3F81),                 # representable
    (1.0 + 2.0 ** -8, 0x3F80),                 # tie, 0x3F80 is even: down
    (1.0 + 3 * 2.0 ** -8, 0x3F82),             # tie, 0x3F81 is odd: up to 0x3F82
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 0x3F81),    # just above the tie: up
    (1.0 + 2.0 ** -8 - 2.0 ** -20, 0x3F80),    # just below the tie: down
    (-(1.0 + 3 * 2.0 ** -8), 0xBF82),          # sign symmetric
    (0.0, 0x0000),
    (-0.0, 0x8000),
    (2.0 ** -133, 0x0001),                     # smallest BF16 subnormal
    (3.0 * 2.0 ** -134, 0x0002),               # subnormal tie 1.5 ulp -> even (2 ulp)
    (from_bits32(0x7F7F7FFF), 0x7F7F),         # below the overflow tie: largest finite
    (from_bits32(0x7F7F8000), 0x7F80),         # overflow tie, 0x7F7F odd: up to +inf
    (1e39, 0x7F80),                            # beyond FP32: +inf
    (-1e39, 0xFF80),
    (math.inf, 0x7F80),
]


@pytest.mark.parametrize("x,expect", BF16_CASES)
def test_bf16_rounding_bits(ora, x, expect):
    got = ora.store_round(2, x)
    b = bits32(got)
    assert b & 0xFFFF == 0, hex(b)             # a BF16 value (low half zero)
    assert b >> 16 == expect, (x, hex(b >> 16), hex(expect))


def test_bf16_nan(ora):
    assert math.isnan(ora.store_round(2, math.nan))


def test_bf16_double_rounding_through_fp32(ora):
    """1 + 2^-8 + 2^-40 lies just above a BF16 tie, but its FP32 rounding is
    the tie itself (2^-40 is below half an FP32 ulp), which then goes to
    even: the stored entry is 1.0, not 1 + 2^-7."""
    assert bits32(ora.store_round(2, 1.0 + 2.0 ** -8 + 2.0 ** -40)) >> 16 == 0x3F80


FP32_CASES = [
    (1.0 + 2.0 ** -24, 0x3F800000),            # tie, even: down
    (1.0 + 3 * 2.0 ** -24, 0x3F800002),        # tie, odd neighbour: up
    (1.0 + 2.0 ** -24 + 2.0 ** -40, 0x3F800001),
    (0.1, 0x3DCCCCCD),
    (-2.0 ** -149, 0x80000001),                # smallest subnormal
    (2.0 ** -150, 0x00000000),                 # tie with zero: even (zero)
    (3.4028234663852886e38, 0x7F7FFFFF),       # FLT_MAX
    (3.4028235677973366e38, 0x7F800000),       # FLT_MAX + half an ulp: the tie goes to +inf
    (1e39, 0x7F800000),
]


@pytest.mark.parametrize("x,expect", FP32_CASES)
def test_fp32_rounding_bits(ora, x, expect):
    assert bits32(ora.store_round(1, x)) == expect, (x, hex(bits32(ora.store_round(1, x))))


def test_fp64_mode_is_identity(ora):
    for x in [0.1, -3.7e-300, 1.0 + 2.0 ** -52]:
        assert ora.store_round(0, x) == x
