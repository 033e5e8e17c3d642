// Elementary functions on the integer pipe for the distribution draws (Sec. 2.4: the
// Gaussian and exponential layers built on the uniform doubles).  The inputs are the
// streams' 48-bit integers, so every step is fixed-point integer arithmetic: on GB300
// the FP64 pipe runs at a small fraction of the integer pipe's rate, and the double
// library functions (log, sqrt, sincospi) bounded the distribution kernels.
//
//  * -ln(w 2^-48): table-driven reduction (Tang, ACM TOMS 16(4), 1990) by a short
//    reciprocal R with m R = 1 - s exact, 0 <= s <= 2^-8.5, then the Taylor series
//    -ln(1 - s) = s q(s), q(s) = sum_j s^j / (j + 1) through j = 6 (remainder
//    < 2^-62), summed in 128-bit fixed point at scale 2^-120.  All coefficients are
//    positive, so every step is an unsigned multiply-high.
//  * sqrt(y): Newton's iteration for 1/sqrt(y) from a single-precision seed, one
//    third-order step t (1 + e/2 + 3e^2/8), e = 1 - y t^2.
//  * cos and sin of 2 pi t for t = v 2^-48 turns: whole quarter turns by swaps and signs,
//    then the nearest first-quadrant table angle j/256 and the remainder beta
//    (|beta| <= 2 pi 2^-9), Taylor series of cos beta and sin beta / beta through
//    beta^6 (remainders < 2^-66), and the angle-sum formulas on magnitudes.
//  * conversion of a 128-bit fixed-point magnitude to the nearest double.
//
// The series coefficients are the exact rationals 1/k, rounded once to the fixed-point
// scale; the tables come from gen_fixmath_tables.py.
#pragma once
#include <cstdint>

#include "rlxpp_fixmath_tables.h"

namespace rlxpp {

struct U128 {
  uint64_t lo, hi;
};

__device__ __forceinline__ U128 mul_wide_u64(uint64_t a, uint64_t b) { return {a * b, __umul64hi(a, b)}; }

__device__ __forceinline__ U128 add_u128(U128 a, U128 b) {
  U128 r;
  asm("add.cc.u64 %0, %2, %4;\n\taddc.u64 %1, %3, %5;"
      : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}
__device__ __forceinline__ U128 sub_u128(U128 a, U128 b) {
  U128 r;
  asm("sub.cc.u64 %0, %2, %4;\n\tsubc.u64 %1, %3, %5;"
      : "=l"(r.lo), "=l"(r.hi) : "l"(a.lo), "l"(a.hi), "l"(b.lo), "l"(b.hi));
  return r;
}

// Rounded fixed-point Taylor coefficient 1/k at scale 2^s.
__host__ __device__ constexpr int64_t fx_inv(int k, int s) { return (int64_t)(((1ull << s) + k / 2) / k); }

// The double nearest to (v.hi 2^64 + v.lo) 2^e (ties to even), negated when neg.  v.hi
// must be nonzero unless v = 0, which gives a zero of that sign; every caller's values
// are 0 or at least 2^72, and the results lie in the normal range.
__device__ __forceinline__ double fx_to_double(U128 v, int e, bool neg) {
  const uint64_t sign = neg ? (1ull << 63) : 0ull;
  const int lz = __clzll((long long)(v.hi | 1));
  const uint64_t top = (v.hi << lz) | ((v.lo >> 1) >> (63 - lz));  // leading 64 bits
  const uint64_t rest = v.lo << lz;
  uint64_t mant = top >> 11;  // 53 bits, leading bit at 52
  mant += ((top >> 10) & 1) & (uint64_t)(((top & 0x3FFull) | rest | (mant & 1)) != 0);
  // v 2^e = (top 2^-63) 2^(127 - lz + e); the leading mantissa bit adds the last unit
  // to the exponent field, and a carry out of the rounding moves to the next binade
  const uint64_t bits = ((uint64_t)(127 - lz + e + 1022) << 52) + mant;
  return __longlong_as_double((long long)((v.hi ? bits : 0ull) | sign));
}

// -ln(w 2^-48) for an integer w in [1, 2^48], at scale 2^-120 (0, or in [2^72, 2^126)).
__device__ __forceinline__ U128 fx_neg_ln48(uint64_t w) {
  const int k = 63 - __clzll((long long)w);      // w = m0 2^k, m0 in [1, 2)
  const uint64_t top = w << (63 - k);             // m0 2^63, at least 15 trailing zeros
  const int up = top > (3ull << 62);              // m0 > 1.5: m = m0 / 2
  const uint64_t M = top >> up;                   // m 2^63, m = w 2^-(k + up) in (0.75, 1.5]
  const ulonglong2 t = __ldg(&kLnTab[((M - 1) >> 54) - 384]);  // interval (i/512, (i+1)/512]
  // m R 2^63 = (M 2^-15) Rint <= 2^63 exactly; s = 1 - m R at scale 2^-64 (< 2^55.5)
  const uint64_t s64 = ((1ull << 63) - (M >> 15) * (t.x & 0xFFFFull)) << 1;
  // q(s) by Horner; the steps j >= 4 are scaled by s^4 < 2^-34 and run in 32 bits at 2^-34
  const uint32_t s40 = (uint32_t)(s64 >> 24);
  uint32_t a = (uint32_t)fx_inv(7, 34);
  a = (uint32_t)fx_inv(6, 34) + (__umulhi(s40, a) >> 8);
  a = (uint32_t)fx_inv(5, 34) + (__umulhi(s40, a) >> 8);
  uint64_t q = (uint64_t)a << 29;                 // scale 2^-63 from here on
  q = (uint64_t)fx_inv(4, 63) + __umul64hi(s64, q);
  q = (uint64_t)fx_inv(3, 63) + __umul64hi(s64, q);
  q = (uint64_t)fx_inv(2, 63) + __umul64hi(s64, q);
  q = (1ull << 63) + __umul64hi(s64, q);
  // -ln(1 - s) = s q at scale 2^-127, to 2^-120
  U128 p = mul_wide_u64(s64, q);
  p = {(p.lo >> 7) | (p.hi << 57), p.hi >> 7};
  // x = (48 - k - up) ln 2 + ln R + s q
  const uint64_t n = (uint64_t)(48 - k - up);
  U128 x = mul_wide_u64(n, kLn2Lo);
  x.hi += n * kLn2Hi;
  x = add_u128(x, U128{t.x & ~0xFFFFull, t.y});
  return add_u128(x, p);
}

// sqrt(2 x) for x = X 2^-120 (X = 0 or X in [2^72, 2^126)), as S 2^se with S in
// [2^60, 2^61), relative error below 2^-59 (the step's remainder (5/16) e^3 < 2^-62 and
// three truncations at 2^-61); X = 0 gives S = 0 through the same steps.
__device__ __forceinline__ uint64_t fx_sqrt2x(U128 X, int& se) {
  const int lz = __clzll((long long)(X.hi | 1));
  uint64_t y = (X.hi << lz) | (X.lo >> (64 - lz));  // the leading 64 bits: 2x = (y 2^-64) 2^(9 - lz)
  int e = 9 - lz;
  if (e & 1) {  // an even exponent: y 2^-64 in [1/4, 1)
    y >>= 1;
    ++e;
  }
  // t = 1/sqrt(y 2^-64) in (1, 2] from single precision (rsqrtf of the leading 24 bits:
  // relative error about 2^-21) as t 2^30 in 32 bits, so that t^2 2^60 is exact in 64
  // and e = 1 - y t^2 exact in 128; then one third-order step, t at scale 2^-61
  const float yf = (float)(uint32_t)(y >> 40) * 0x1p-24f;
  const uint64_t t30 = __float2uint_rn(rsqrtf(yf) * 0x1p30f);
  const U128 d = sub_u128(U128{0, 1ull << 60}, mul_wide_u64(y, t30 * t30));  // e 2^124
  const int64_t e80 = (int64_t)((d.lo >> 44) | (d.hi << 20));              // |e| < 2^-19
  const int64_t c80 = e80 / 2 + ((__mul64hi(e80, e80) * 3) >> 19);         // e/2 + 3e^2/8
  const uint64_t t0 = t30 << 31;
  const uint64_t t1 = t0 + (uint64_t)(__mul64hi((int64_t)t0, c80) >> 16);   // t c at 2^-77, to 2^-61
  se = e / 2 - 61;
  return __umul64hi(y, t1);  // sqrt(y 2^-64) 2^61
}

// cos and sin of 2 pi v 2^-48 (v < 2^48): magnitudes at scale 2^-62 (absolute error below
// 2^-59) and signs.
struct FxCosSin {
  uint64_t c, s;
  bool nc, ns;
};
__device__ __forceinline__ FxCosSin fx_cos_sin_2pi48(uint64_t v) {
  const uint32_t quad = (uint32_t)(v >> 46);                 // whole quarter turns
  const uint64_t f = v & ((1ull << 46) - 1);                 // the rest, under a quarter
  const uint64_t j = (f + (1ull << 39)) >> 40;               // nearest j / 256, 0..64
  const int64_t b = (int64_t)f - (int64_t)(j << 40);        // remainder b 2^-48 turns, |b| <= 2^39
  const ulonglong2 sc = __ldg(&kSinCosTab[j]);              // sin, cos of 2 pi j / 256 at 2^-63
  const U128 pb = mul_wide_u64((uint64_t)(b < 0 ? -b : b), kTwoPi61);  // |beta| 2^109
  const uint64_t beta69 = (pb.lo >> 40) | (pb.hi << 24);    // |beta| 2^69 < 2^63
  const uint64_t s74 = __umul64hi(beta69, beta69);          // s = beta^2, at 2^-74 (< 2^61.3)
  // cos beta = 1 - s (1/2 - s (1/24 - s/720)) and sin beta / beta = 1 - s (1/6 - s (1/120 -
  // s/5040)); the innermost brackets are scaled by s^2 < 2^-25 and run in 32 bits at 2^-36
  const uint32_t s42 = (uint32_t)(s74 >> 32);
  const uint64_t ic = (uint64_t)((uint32_t)fx_inv(24, 36) - (__umulhi(s42, (uint32_t)fx_inv(720, 36)) >> 10)) << 27;
  const uint64_t is = (uint64_t)((uint32_t)fx_inv(120, 36) - (__umulhi(s42, (uint32_t)fx_inv(5040, 36)) >> 10)) << 27;
  const uint64_t mc = (uint64_t)fx_inv(2, 63) - (__umul64hi(s74, ic) >> 10);
  const uint64_t ms = (uint64_t)fx_inv(6, 63) - (__umul64hi(s74, is) >> 10);
  const uint64_t cb = (1ull << 63) - (__umul64hi(s74, mc) >> 10);               // cos beta 2^63
  const uint64_t sb = __umul64hi(beta69, (1ull << 63) - (__umul64hi(s74, ms) >> 10)) >> 5;  // |sin beta| 2^63
  // the first-quadrant angle sums, at 2^-62
  const uint64_t scb = __umul64hi(sc.x, cb), ccb = __umul64hi(sc.y, cb);
  const uint64_t csb = __umul64hi(sc.y, sb), ssb = __umul64hi(sc.x, sb);
  const uint64_t sa = b < 0 ? scb - csb : scb + csb;
  const uint64_t ca = b < 0 ? ccb + ssb : ccb - ssb;
  // quarter turns: (c, s) -> (-s, c)
  FxCosSin r;
  r.c = (quad & 1) ? sa : ca;
  r.s = (quad & 1) ? ca : sa;
  r.nc = quad == 1 || quad == 2;
  r.ns = quad >= 2;
  return r;
}

// s 2^se times m 2^-62 as a double, negated when neg (s = 0 or s >= 2^60; m = 0 or m >= 2^12).
__device__ __forceinline__ double fx_scale_to_double(uint64_t s, int se, uint64_t m, bool neg) {
  return fx_to_double(mul_wide_u64(s, m), se - 62, neg);
}

// Exponential value -ln(1 - v 2^-48) for a 48-bit v.
__device__ __forceinline__ double fx_exponential48(uint64_t v) {
  return fx_to_double(fx_neg_ln48((1ull << 48) - v), -120, false);
}

// Box-Muller pair from 48-bit va, vb: r = sqrt(-2 ln(1 - va 2^-48)), (r cos 2 pi vb 2^-48,
// r sin 2 pi vb 2^-48).
__device__ __forceinline__ void fx_box_muller48(uint64_t va, uint64_t vb, double& z0, double& z1) {
  int se;
  const uint64_t s = fx_sqrt2x(fx_neg_ln48((1ull << 48) - va), se);
  const FxCosSin cs = fx_cos_sin_2pi48(vb);
  z0 = fx_scale_to_double(s, se, cs.c, cs.nc);
  z1 = fx_scale_to_double(s, se, cs.s, cs.ns);
}

}  // namespace rlxpp
