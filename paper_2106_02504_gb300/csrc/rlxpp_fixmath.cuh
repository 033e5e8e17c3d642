// Elementary functions on the integer pipe for the distribution draws (Sec. 2.4: the
// Gaussian and exponential layers built on the uniform doubles).  The inputs are the
// streams' 48-bit integers, so every step is fixed-point integer arithmetic: on GB300
// the FP64 pipe runs at a small fraction of the integer pipe's rate, and the double
// library functions (log, sqrt, sincospi) bounded the distribution kernels.
//
//  * -ln(w 2^-48): table-driven reduction (Tang, ACM TOMS 16(4), 1990) by a short
//    reciprocal R with m R = 1 + r exact, |r| <= 2^-8, then the Taylor series
//    ln(1 + r) = r q(r), q(r) = sum_j (-r)^j / (j + 1) through j = 7 (remainder
//    < 2^-66), summed in 128-bit fixed point at scale 2^-120.
//  * sqrt(y): Newton's iteration for 1/sqrt(y) from a single-precision seed, one
//    third-order step t (1 + e/2 + 3e^2/8), e = 1 - y t^2.
//  * cos and sin of 2 pi t for t = v 2^-48 turns: nearest table angle j/256 and the
//    remainder beta (|beta| <= 2 pi 2^-9), Taylor series of cos beta and sin beta / beta
//    through beta^6 (remainders < 2^-66), then the angle-sum formulas.
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

// The double nearest to (v.hi 2^64 + v.lo) 2^e, negated when neg (ties to even); v = 0
// gives a zero of that sign.  The result must lie in the normal range (every caller
// keeps it within 2^-130 .. 2^10).
__device__ __forceinline__ double fx_to_double(U128 v, int e, bool neg) {
  const uint64_t sign = neg ? (1ull << 63) : 0ull;
  if ((v.hi | v.lo) == 0) return __longlong_as_double((long long)sign);
  const int lz = v.hi ? __clzll((long long)v.hi) : 64 + __clzll((long long)v.lo);
  uint64_t top, rest;  // v 2^lz = top 2^64 + rest, top in [2^63, 2^64)
  if (lz == 0) {
    top = v.hi;
    rest = v.lo;
  } else if (lz < 64) {
    top = (v.hi << lz) | (v.lo >> (64 - lz));
    rest = v.lo << lz;
  } else {
    top = v.lo << (lz - 64);
    rest = 0;
  }
  uint64_t mant = top >> 11;  // 53 bits, leading bit at 52
  const bool up = ((top >> 10) & 1) && ((top & 0x3FFull) | rest | (mant & 1));
  mant += up;
  const int lead = 127 - lz + e;  // v 2^e = (top 2^-63) 2^lead
  // the leading mantissa bit adds the last unit to the exponent field; a carry out of
  // the rounding moves to the next binade by the same addition
  const uint64_t bits = ((uint64_t)(lead + 1022) << 52) + mant;
  return __longlong_as_double((long long)(bits | sign));
}

// -ln(w 2^-48) for an integer w in [1, 2^48], at scale 2^-120 (< 2^126).
__device__ __forceinline__ U128 fx_neg_ln48(uint64_t w) {
  const int k = 63 - __clzll((long long)w);             // w = m0 2^k, m0 in [1, 2)
  const int kk = k + (int)(((w << (63 - k)) >> 62) & 1);  // m = w 2^-kk in [0.75, 1.5)
  const int i = (int)((w << (62 - kk)) >> 54);          // floor(256 m), 192..383
  const ulonglong2 t = __ldg(&kLnTab[i - 192]);
  const uint64_t rint = t.x & 0x1FFFull;                 // R = rint / 4096
  // (1 + r) 2^61 = m R 2^61 = w rint 2^(49 - kk), exact (w rint < 2^61)
  const int64_t r61 = (int64_t)((w * rint) << (49 - kk)) - (1ll << 61);
  const int64_t r70 = r61 * 512;                         // r 2^70, |r| <= 2^-8
  // q(r) by Horner: the terms j >= 4 only need 2^-30 (they are scaled by r^4 <= 2^-32)
  const int32_t r38 = (int32_t)(r70 >> 32);
  int32_t a = (int32_t)-fx_inv(8, 30);
  a = (int32_t)fx_inv(7, 30) + (__mulhi(r38, a) >> 6);
  a = (int32_t)-fx_inv(6, 30) + (__mulhi(r38, a) >> 6);
  a = (int32_t)fx_inv(5, 30) + (__mulhi(r38, a) >> 6);
  int64_t q = (int64_t)a * (1ll << 32);                  // scale 2^-62 from here on
  q = -fx_inv(4, 62) + (__mul64hi(r70, q) >> 6);
  q = fx_inv(3, 62) + (__mul64hi(r70, q) >> 6);
  q = -fx_inv(2, 62) + (__mul64hi(r70, q) >> 6);
  q = (1ll << 62) + (__mul64hi(r70, q) >> 6);
  // ln(1 + r) = r q at scale 2^-123, as a magnitude; to 2^-120
  const uint64_t ar = (uint64_t)(r61 < 0 ? -r61 : r61);
  U128 p = mul_wide_u64(ar, (uint64_t)q);
  p = {(p.lo >> 3) | (p.hi << 61), p.hi >> 3};
  // x = (48 - kk) ln 2 + ln R - ln(1 + r)
  const uint64_t n = (uint64_t)(48 - kk);
  U128 x = mul_wide_u64(n, kLn2Lo);
  x.hi += n * kLn2Hi;
  x = add_u128(x, U128{t.x & ~0x1FFFull, t.y});
  return r61 < 0 ? add_u128(x, p) : sub_u128(x, p);
}

// sqrt(2 x) for x = X 2^-120 (X < 2^126), as S 2^se with S in [2^60, 2^61), relative
// error below 2^-59 (the step's remainder (5/16) e^3 < 2^-62 and three truncations at
// 2^-61); S = 0 for X = 0.
__device__ __forceinline__ uint64_t fx_sqrt2x(U128 X, int& se) {
  if ((X.hi | X.lo) == 0) {
    se = 0;
    return 0;
  }
  const int lz = X.hi ? __clzll((long long)X.hi) : 64 + __clzll((long long)X.lo);
  uint64_t y;  // the leading 64 bits of X: 2x = (y 2^-64) 2^(9 - lz)
  if (lz == 0) y = X.hi;
  else if (lz < 64) y = (X.hi << lz) | (X.lo >> (64 - lz));
  else y = X.lo << (lz - 64);
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
  return __umul64hi(y, t1);                                 // sqrt(y 2^-64) 2^61
}

// cos and sin of 2 pi v 2^-48 (v < 2^48) at scale 2^-60, absolute error below 2^-57.
__device__ __forceinline__ void fx_cos_sin_2pi48(uint64_t v, int64_t& c60, int64_t& s60) {
  const uint64_t jj = (v + (1ull << 39)) >> 40;             // nearest j / 256, 0..256
  const int64_t b = (int64_t)v - (int64_t)(jj << 40);      // remainder b 2^-48 turns, |b| <= 2^39
  const longlong2 sc = __ldg(&kSinCosTab[jj & 255]);
  const uint64_t ab = (uint64_t)(b < 0 ? -b : b);
  const U128 pb = mul_wide_u64(ab, kTwoPi61);               // |beta| 2^109
  const uint64_t beta69 = (pb.lo >> 40) | (pb.hi << 24);    // |beta| 2^69 < 2^63
  const int64_t s74 = (int64_t)__umul64hi(beta69, beta69);  // beta^2 2^74
  // cos beta = 1 - s/2 + s^2/24 - s^3/720, sin beta / beta = 1 - s/6 + s^2/120 - s^3/5040
  int64_t qc = -fx_inv(720, 62);
  qc = fx_inv(24, 62) + (__mul64hi(s74, qc) >> 10);
  qc = -fx_inv(2, 62) + (__mul64hi(s74, qc) >> 10);
  qc = (1ll << 62) + (__mul64hi(s74, qc) >> 10);
  int64_t ps = -fx_inv(5040, 62);
  ps = fx_inv(120, 62) + (__mul64hi(s74, ps) >> 10);
  ps = -fx_inv(6, 62) + (__mul64hi(s74, ps) >> 10);
  ps = (1ll << 62) + (__mul64hi(s74, ps) >> 10);
  int64_t sb = (int64_t)(__umul64hi(beta69, (uint64_t)ps) >> 5);  // |sin beta| 2^62
  if (b < 0) sb = -sb;
  // angle sums with the table's sin(2 pi j/256) (x) and cos(2 pi j/256) (y)
  s60 = __mul64hi(sc.x, qc) + __mul64hi(sc.y, sb);
  c60 = __mul64hi(sc.y, qc) - __mul64hi(sc.x, sb);
}

// s 2^se times c 2^-60 as a double (s < 2^61, |c| <= 2^60).
__device__ __forceinline__ double fx_scale_to_double(uint64_t s, int se, int64_t c) {
  const uint64_t ac = (uint64_t)(c < 0 ? -c : c);
  return fx_to_double(mul_wide_u64(s, ac), se - 60, c < 0);
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
  int64_t c, sn;
  fx_cos_sin_2pi48(vb, c, sn);
  z0 = fx_scale_to_double(s, se, c);
  z1 = fx_scale_to_double(s, se, sn);
}

}  // namespace rlxpp
