"""Writes rlxpp_fixmath_tables.h: the constant tables of the integer-pipe elementary
functions in rlxpp_fixmath.cuh, computed with Python's decimal module at 90 digits and
rounded once to the stored fixed-point scale.

  * ln 2 at scale 2^-120 (128 bits) and 2 pi at scale 2^-61 (64 bits);
  * the logarithm's reduction table (table-driven logarithm, Tang, ACM TOMS 16(4),
    1990): for the mantissa interval (i/512, (i+1)/512], i = 384..767, the 16-bit
    reciprocal R_i = Rint_i / 2^15 of the interval's upper end, rounded down (so that
    m R_i <= 1 on the interval; exactly 1 for the interval ending at 1), and ln R_i at
    scale 2^-120, rounded to a multiple of 2^16 so that Rint_i fits in the low 16 bits
    of the same 128-bit word;
  * sin and cos of 2 pi j / 256 for the first quadrant, j = 0..64, at scale 2^-63.

Run it from anywhere: ``python gen_fixmath_tables.py`` rewrites the header beside it.
"""
from __future__ import annotations

import os
from decimal import Decimal, ROUND_HALF_EVEN, getcontext

getcontext().prec = 90
EPS = Decimal(10) ** -88


def atan_inv(k):
    """arctan(1/k) by its Taylor series (k > 1)."""
    x = Decimal(1) / k
    x2 = x * x
    term, total, n, sign = x, Decimal(0), 1, 1
    while term > EPS:
        total += sign * term / n
        term *= x2
        n += 2
        sign = -sign
    return total


PI = 16 * atan_inv(5) - 4 * atan_inv(239)        # Machin's formula


def sin_cos(theta):
    """(sin, cos) of theta by their Taylor series, after reducing theta into [-pi, pi]."""
    two_pi = 2 * PI
    theta = theta - two_pi * (theta / two_pi).to_integral_value(rounding=ROUND_HALF_EVEN)
    s, c = Decimal(0), Decimal(0)
    term, n = Decimal(1), 0                    # term = theta^n / n!
    while abs(term) > EPS or n < 4:
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * theta / n
    return s, c


def fixed(x, scale_bits):
    return int((x * (Decimal(2) ** scale_bits)).to_integral_value(rounding=ROUND_HALF_EVEN))


def ln_table():
    rows = []
    for i in range(384, 768):
        rint = (1 << 15) * 512 // (i + 1)           # floor(2^15 / upper end)
        # r = m R - 1 lies in [-2^-8.5, 0] over the interval (the series' range)
        for m in (Decimal(i) / 512, Decimal(i + 1) / 512):
            r = m * rint / (1 << 15) - 1
            assert -Decimal(2) ** Decimal("-8.5") <= r <= 0, (i, rint)
        assert 0 < rint < 1 << 16
        v = fixed((Decimal(rint) / (1 << 15)).ln(), 120)
        v = (v + (1 << 15)) >> 16 << 16                # a multiple of 2^16
        v &= (1 << 128) - 1                             # two's complement, 128 bits
        rows.append(((v & ((1 << 64) - 1)) | rint, v >> 64))
    return rows


def sincos_table():
    rows = []
    for j in range(65):
        s, c = sin_cos(2 * PI * j / 256)
        rows.append((fixed(s, 63), fixed(c, 63)))
    return rows


def render():
    ln2 = fixed(Decimal(2).ln(), 120)
    two_pi = fixed(2 * PI, 61)
    assert ln2 < 1 << 128 and two_pi < 1 << 64
    out = ["// Generated by gen_fixmath_tables.py (decimal arithmetic at 90 digits); do not edit.",
           "#pragma once", "#include <cstdint>", "", "namespace rlxpp {", "",
           "// ln 2 2^120 as (low, high) 64-bit words; 2 pi 2^61.",
           f"constexpr uint64_t kLn2Lo = 0x{ln2 & ((1 << 64) - 1):016x}ull;",
           f"constexpr uint64_t kLn2Hi = 0x{ln2 >> 64:016x}ull;",
           f"constexpr uint64_t kTwoPi61 = 0x{two_pi:016x}ull;", "",
           "// Logarithm reduction, i = 384..767 (mantissa in (i/512, (i+1)/512]): x = low word",
           "// with the reciprocal numerator Rint (R = Rint / 2^15) in bits 0..15, y = high word;",
           "// with those 16 bits cleared, (y:x) is ln R 2^120 in two's complement.",
           "static __device__ const ulonglong2 kLnTab[384] = {"]
    for lo, hi in ln_table():
        out.append(f"    {{0x{lo:016x}ull, 0x{hi:016x}ull}},")
    out += ["};", "",
            "// sin(2 pi j / 256) 2^63 and cos(2 pi j / 256) 2^63, j = 0..64 (the first quadrant).",
            "static __device__ const ulonglong2 kSinCosTab[65] = {"]
    for s, c in sincos_table():
        out.append(f"    {{0x{s:016x}ull, 0x{c:016x}ull}},")
    out += ["};", "", "}  // namespace rlxpp", ""]
    return "\n".join(out)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rlxpp_fixmath_tables.h")
    with open(path, "w") as f:
        f.write(render())
    print(path)
