// 576-bit modular arithmetic for RANLUX++ on sm_103a: the LCG advance X <- A X mod m
// with m = 2^576 - 2^240 + 1 (Sec. 2.2 of Hahnfeld & Moneta, arXiv 2106.02504), the
// 576 x 576 -> 1152-bit product (Sec. 2.1), the reduction mod m (Sec. 2.2) and the
// conversion between the LCG state and the 24 RANLUX numbers (Sec. 2.3).
//
// Numbers are little-endian arrays of 32-bit limbs held in registers: 18 limbs for a
// 576-bit value, 36 for a product.  Carry chains are written with PTX add.cc/addc
// (the GPU counterpart of the branch-free carry propagation of Sec. 3.4) and the limb
// products with mad.wide.u32 (32 x 32 -> 64 bits, the device has no 128-bit integer
// type; Sec. 4.2).  Every loop has a compile-time trip count and is fully unrolled
// (Sec. 3.1).
#pragma once
#include <cstdint>

namespace rlxpp {

constexpr int kLimbs = 18;        // 576 / 32
constexpr int kWords = 24;        // RANLUX numbers per block
constexpr int kDoubles = 12;      // 48-bit doubles per block

// ---------------------------------------------------------------------------------
// carry-chain primitives (PTX condition-code chains; kept in program order by volatile)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t add_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t addc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("addc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t sub_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("sub.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t subc_cc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.cc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t subc(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("subc.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c) {
  uint64_t r;
  asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(r) : "r"(a), "r"(b), "l"(c));
  return r;
}
__device__ __forceinline__ uint32_t lo32(uint64_t v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t hi32(uint64_t v) { return (uint32_t)(v >> 32); }
// (hi:lo) >> s for 0 < s < 32
__device__ __forceinline__ uint32_t shr_pair(uint32_t lo, uint32_t hi, int s) {
  return __funnelshift_r(lo, hi, s);
}

// ---------------------------------------------------------------------------------
// Sec. 2.1: the 576 x 576 -> 1152-bit product.
//
// mul_9x9 multiplies two 9-limb (288-bit) numbers by operand scanning: row i adds
// a_i * b shifted by i limbs; the 9 products a_i b_j + p_{i+j} fit in 64 bits each
// ((2^32-1)^2 + 2^32-1 < 2^64) and are independent, and one carry chain adds the high
// half of product j-1 to the low half of product j.  After row i the partial product
// (a mod 2^(32(i+1))) b fits in limbs 0..i+9, so no carry leaves limb i+9.
// The multiplier comes through an accessor so that a constant can stay in the constant
// bank (kernel parameters) instead of registers.
// ---------------------------------------------------------------------------------
template <class AFn>
__device__ __forceinline__ void mul_9x9(AFn a, const uint32_t* b, uint32_t* p) {
#pragma unroll
  for (int k = 0; k < 18; ++k) p[k] = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const uint32_t ai = a(i);
    uint64_t t[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) t[j] = mad_wide(ai, b[j], (uint64_t)p[i + j]);
    p[i] = lo32(t[0]);
    p[i + 1] = add_cc(lo32(t[1]), hi32(t[0]));
#pragma unroll
    for (int j = 2; j < 9; ++j) p[i + j] = addc_cc(lo32(t[j]), hi32(t[j - 1]));
    p[i + 9] = addc(hi32(t[8]), 0u);
  }
}

// multiply9x9 with one level of Karatsuba (243 limb products instead of 324).  With
// A = A1 2^288 + A0 and X = X1 2^288 + X0,
//   A X = A1 X1 2^576 + ((A0 + A1)(X0 + X1) - A0 X0 - A1 X1) 2^288 + A0 X0.
// The half sums carry one extra bit each: A0 + A1 = As + ca 2^288, X0 + X1 = Xs + cx 2^288,
// so (A0 + A1)(X0 + X1) = As Xs + 2^288 (cx As + ca Xs) + ca cx 2^576 (below 2^578).
// a(i), i < 18: limbs of A; as(i), i < 9: limbs of As; ca: its carry.
template <class AFn, class ASFn>
__device__ __forceinline__ void multiply9x9_split(AFn a, ASFn as, uint32_t ca, const uint32_t X[kLimbs],
                                                  uint32_t P[2 * kLimbs]) {
  uint32_t Xs[9];
  Xs[0] = add_cc(X[0], X[9]);
#pragma unroll
  for (int k = 1; k < 9; ++k) Xs[k] = addc_cc(X[k], X[9 + k]);
  const uint32_t cx = addc(0u, 0u);
  uint32_t P0[18], P2[18], M[20];
  mul_9x9([&](int i) { return a(i); }, X, P0);
  mul_9x9([&](int i) { return a(9 + i); }, X + 9, P2);
  mul_9x9(as, Xs, M);
  // M += 2^288 (cx As + ca Xs) + ca cx 2^576
  const uint32_t mx = 0u - cx;
  M[9] = add_cc(M[9], as(0) & mx);
#pragma unroll
  for (int k = 1; k < 9; ++k) M[9 + k] = addc_cc(M[9 + k], as(k) & mx);
  M[18] = addc(0u, 0u);
  M[19] = 0u;
  if (ca) {
    M[9] = add_cc(M[9], Xs[0]);
#pragma unroll
    for (int k = 1; k < 9; ++k) M[9 + k] = addc_cc(M[9 + k], Xs[k]);
    M[18] = addc_cc(M[18], cx);
    M[19] = addc(0u, 0u);
  }
  // middle term M - A0 X0 - A1 X1 (non-negative, 20 limbs)
  M[0] = sub_cc(M[0], P0[0]);
#pragma unroll
  for (int k = 1; k < 18; ++k) M[k] = subc_cc(M[k], P0[k]);
  M[18] = subc_cc(M[18], 0u);
  M[19] = subc(M[19], 0u);
  M[0] = sub_cc(M[0], P2[0]);
#pragma unroll
  for (int k = 1; k < 18; ++k) M[k] = subc_cc(M[k], P2[k]);
  M[18] = subc_cc(M[18], 0u);
  M[19] = subc(M[19], 0u);
  // P = A0 X0 + A1 X1 2^576 + middle 2^288
#pragma unroll
  for (int k = 0; k < 18; ++k) {
    P[k] = P0[k];
    P[18 + k] = P2[k];
  }
  P[9] = add_cc(P[9], M[0]);
#pragma unroll
  for (int k = 1; k < 20; ++k) P[9 + k] = addc_cc(P[9 + k], M[k]);
#pragma unroll
  for (int k = 29; k < 35; ++k) P[k] = addc_cc(P[k], 0u);
  P[35] = addc(P[35], 0u);
}

// Both operands variable: the half sum of A is formed here.
template <class AFn>
__device__ __forceinline__ void multiply9x9(AFn a, const uint32_t X[kLimbs], uint32_t P[2 * kLimbs]) {
  uint32_t As[9];
  As[0] = add_cc(a(0), a(9));
#pragma unroll
  for (int k = 1; k < 9; ++k) As[k] = addc_cc(a(k), a(9 + k));
  const uint32_t ca = addc(0u, 0u);
  multiply9x9_split(a, [&](int i) { return As[i]; }, ca, X, P);
}

// ---------------------------------------------------------------------------------
// Sec. 2.2: r = p mod m, m = 2^576 - 2^240 + 1, using only additions, subtractions and
// shifts, with the final correction that puts the result in [0, m).
//
// With 2^576 = 2^240 - 1 (mod m), write p = H 2^576 + L and H = H1 2^336 + H0:
//   p = L + H 2^240 - H = L + H0 2^240 + H1 2^576 - H = L + (H0 + H1) 2^240 - H - H1.
// Adding 2m keeps every intermediate non-negative:
//   R = L + S 2^240 + (2m - V),  S = H0 + H1 < 2^337,  V = H + H1 < 2m,
// so 0 <= R < 5 2^576.  Folding the top limb t (0..4) with 2^576 = 2^240 - 1 leaves at
// most one more 2^576 overflow c, and when c = 1 the low part is below 2^243, so the
// second fold only touches limbs 0..7.  The result is then below 2^576 and at most one
// subtraction of m puts it in [0, m): r >= m exactly when r + (2^240 - 1) >= 2^576.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void mod_m(const uint32_t p[2 * kLimbs], uint32_t r[kLimbs]) {
  const uint32_t* L = p;
  const uint32_t* H = p + kLimbs;
  // H1 = H >> 336 (240 bits, limbs 0..7; limb 7 holds 16 bits)
  uint32_t H1[8];
#pragma unroll
  for (int k = 0; k < 7; ++k) H1[k] = shr_pair(H[10 + k], H[11 + k], 16);
  H1[7] = H[17] >> 16;
  // V = H + H1 (19 limbs, top limb 0 or 1) and S = H0 + H1, H0 = H mod 2^336 (limbs
  // 0..9 and the low 16 bits of limb 10), agree in limbs 0..9, whose sum is formed
  // once.  H1 < 2^240, so a carry out of limb 7 needs limbs 0..7 of H within H1 of 2^256
  // (about 2^-16 of the products): only then do the chains go on.
  uint32_t V[kLimbs + 1];
  V[0] = add_cc(H[0], H1[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) V[k] = addc_cc(H[k], H1[k]);
  const uint32_t c8 = addc(0u, 0u);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) V[k] = H[k];
  V[kLimbs] = 0u;
  uint32_t S10 = H[10] & 0xFFFFu;  // limb 10 of S
  if (__builtin_expect(c8 != 0u, 0)) {
    V[8] = add_cc(H[8], 1u);
#pragma unroll
    for (int k = 9; k < kLimbs; ++k) V[k] = addc_cc(H[k], 0u);
    V[kLimbs] = addc(0u, 0u);
    // the carry leaves limb 9 exactly when limbs 8 and 9 were all ones (both now zero)
    S10 += (V[8] | V[9]) == 0u ? 1u : 0u;
  }
  // W = 2m - V; 2m = 2^577 - 2^241 + 2: limb 0 = 2, limb 7 = 0xFFFE0000,
  // limbs 8..17 = 0xFFFFFFFF, limb 18 = 1, other limbs 0.
  uint32_t W[kLimbs + 1];
  W[0] = sub_cc(2u, V[0]);
#pragma unroll
  for (int k = 1; k < 7; ++k) W[k] = subc_cc(0u, V[k]);
  W[7] = subc_cc(0xFFFE0000u, V[7]);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) W[k] = subc_cc(0xFFFFFFFFu, V[k]);
  W[kLimbs] = subc(1u, V[kLimbs]);
  // U = L + (S << 240); 240 = 7 limbs + 16 bits, S << 240 covers limbs 7..18
  uint32_t Sh[12];
  Sh[0] = V[0] << 16;
#pragma unroll
  for (int k = 1; k < 10; ++k) Sh[k] = __funnelshift_l(V[k - 1], V[k], 16);
  Sh[10] = __funnelshift_l(V[9], S10, 16);
  Sh[11] = S10 >> 16;
  uint32_t R[kLimbs + 1];
  // R = L + W first (limbs 0..6 of the shifted S are zero), then add the shifted S.
  R[0] = add_cc(L[0], W[0]);
#pragma unroll
  for (int k = 1; k < kLimbs; ++k) R[k] = addc_cc(L[k], W[k]);
  R[kLimbs] = addc(W[kLimbs], 0u);
  R[7] = add_cc(R[7], Sh[0]);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) R[k] = addc_cc(R[k], Sh[k - 7]);
  R[kLimbs] = addc(R[kLimbs], Sh[11]);
  // fold 1: R = R[0..17] + t (2^240 - 1), t = R[18] in 0..4.
  // t (2^240 - 1) = t 2^240 - t: limbs 0..6 of (2^240 - t) and limb 7 = (t - 1) 2^16 + 0xFFFF
  // for t >= 1; all zero for t = 0.
  const uint32_t t = R[kLimbs];
  const uint32_t nz = t ? 0xFFFFFFFFu : 0u;
  r[0] = add_cc(R[0], (0u - t));
#pragma unroll
  for (int k = 1; k < 7; ++k) r[k] = addc_cc(R[k], nz);
  r[7] = addc_cc(R[7], ((t - 1u) << 16 | 0xFFFFu) & nz);
  const uint32_t f8 = addc(0u, 0u);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) r[k] = R[k];
  // t (2^240 - 1) < 2^243, so a carry out of limb 7 is rare (at most about 2^-13), and
  // only then does the chain go on.  fold 2: a carry c out of limb 17 adds c (2^240 - 1);
  // when c = 1 the value is below 2^243, so that addition stops at limb 7.
  if (__builtin_expect(f8 != 0u, 0)) {
    r[8] = add_cc(R[8], 1u);
#pragma unroll
    for (int k = 9; k < kLimbs; ++k) r[k] = addc_cc(R[k], 0u);
    if (addc(0u, 0u)) {
      r[0] = add_cc(r[0], 0xFFFFFFFFu);
#pragma unroll
      for (int k = 1; k < 7; ++k) r[k] = addc_cc(r[k], 0xFFFFFFFFu);
      r[7] = addc(r[7], 0xFFFFu);
    }
  }
  // final correction: r >= m  <=>  r + (2^240 - 1) >= 2^576; then r - m = that sum mod
  // 2^576.  r >= m needs bits 240..575 of r all set: the top limb is tested first.
  if (__builtin_expect(r[17] == 0xFFFFFFFFu, 0)) {
    const uint32_t top = r[8] & r[9] & r[10] & r[11] & r[12] & r[13] & r[14] & r[15] & r[16];
    if (top == 0xFFFFFFFFu && r[7] >= 0xFFFF0000u) {
      uint32_t e[kLimbs];
      e[0] = add_cc(r[0], 0xFFFFFFFFu);
#pragma unroll
      for (int k = 1; k < 7; ++k) e[k] = addc_cc(r[k], 0xFFFFFFFFu);
      e[7] = addc_cc(r[7], 0xFFFFu);
#pragma unroll
      for (int k = 8; k < kLimbs; ++k) e[k] = addc_cc(r[k], 0u);
      const uint32_t ge = addc(0u, 0u);
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) r[k] = ge ? e[k] : r[k];
    }
  }
}

// ---------------------------------------------------------------------------------
// Sec. 2.3: LCG state X (in [0, m)) -> the 24 RANLUX numbers D = floor(2^576 X / m).
// 2^576 = m + 2^240 - 1 gives D = X + q with q = floor(T / m), T = X (2^240 - 1) < 2^816.
// Since m < 2^576 and T / m - T / 2^576 < 2^-96, q is q0 = floor(T / 2^576) or q0 + 1,
// and q = q0 + 1 exactly when (q0 + 1) m <= T, i.e. when
//   T_lo + (q0 + 1)(2^240 - 1) >= 2^576,  T_lo = T mod 2^576,
// using (q0 + 1) m = (q0 + 1) 2^576 - (q0 + 1)(2^240 - 1).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void to_ranlux_full(const uint32_t X[kLimbs], uint32_t D[kLimbs]) {
  // T = (X << 240) - X, 26 limbs
  uint32_t T[26];
  T[0] = sub_cc(0u, X[0]);
#pragma unroll
  for (int k = 1; k < 7; ++k) T[k] = subc_cc(0u, X[k]);
  T[7] = subc_cc(X[0] << 16, X[7]);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) T[k] = subc_cc(__funnelshift_l(X[k - 8], X[k - 7], 16), X[k]);
#pragma unroll
  for (int k = kLimbs; k < 25; ++k) T[k] = subc_cc(__funnelshift_l(X[k - 8], X[k - 7], 16), 0u);
  T[25] = subc(X[17] >> 16, 0u);
  // q = q0 + 1 needs T_lo + (q0 + 1)(2^240 - 1) >= 2^576 with (q0 + 1)(2^240 - 1) < 2^480,
  // so T_lo must have bits 480..575 all set (limbs 15..17 all ones); only then is the
  // exact test run (probability about 2^-96 for a random state).
  if ((T[15] & T[16] & T[17]) == 0xFFFFFFFFu) {
    uint32_t q1[8];  // q0 + 1 (q0 = T >> 576, limbs 18..25, below 2^240)
    q1[0] = add_cc(T[18], 1u);
#pragma unroll
    for (int k = 1; k < 8; ++k) q1[k] = addc_cc(T[18 + k], 0u);
    // F = T_lo - q1 + (q1 << 240): compare against 2^576 through the net carry
    uint32_t F[kLimbs];
    F[0] = sub_cc(T[0], q1[0]);
#pragma unroll
    for (int k = 1; k < 8; ++k) F[k] = subc_cc(T[k], q1[k]);
#pragma unroll
    for (int k = 8; k < kLimbs; ++k) F[k] = subc_cc(T[k], 0u);
    const uint32_t borrow = subc(0u, 0u);  // 0 or 0xFFFFFFFF
    // q1 << 240 occupies limbs 7..15 (q1 <= 2^240): limb 7 + k holds the top 16 bits of
    // q1[k-1] and the low 16 bits of q1[k], limb 15 the top 16 bits of q1[7].
    uint32_t dummy = add_cc(F[7], q1[0] << 16);
#pragma unroll
    for (int k = 8; k < 15; ++k) dummy = addc_cc(F[k], __funnelshift_l(q1[k - 8], q1[k - 7], 16));
    dummy = addc_cc(F[15], q1[7] >> 16);
    dummy = addc_cc(F[16], 0u);
    dummy = addc_cc(F[17], 0u);
    (void)dummy;
    const uint32_t carry = addc(0u, 0u);
    // overflow of F past 2^576 = carry - borrow bit; q = q0 + 1 iff it is +1
    if (carry == 1u && borrow == 0u) {
#pragma unroll
      for (int k = 0; k < 8; ++k) T[18 + k] = q1[k];
    }
  }
  D[0] = add_cc(X[0], T[18]);
#pragma unroll
  for (int k = 1; k < 8; ++k) D[k] = addc_cc(X[k], T[18 + k]);
#pragma unroll
  for (int k = 8; k < kLimbs - 1; ++k) D[k] = addc_cc(X[k], 0u);
  D[kLimbs - 1] = addc(X[kLimbs - 1], 0u);
}

// The same D with the long chain only where it decides anything.  T = X 2^240 - X has
// T_lo = (S - X) mod 2^576 with S = (X << 240) mod 2^576, and q0 = (X >> 336) - [S < X].
// The top three limbs of S - X, taken without the borrow from limb 14, settle both
// [S < X] (their own borrow) and that q = q0 (T_lo is not all ones in limbs 15..17)
// unless they are all zeros or all ones, about 2^-95 of the inputs; those go through
// to_ranlux_full.
__device__ __forceinline__ void to_ranlux(const uint32_t X[kLimbs], uint32_t D[kLimbs]) {
  const uint32_t t15 = sub_cc(__funnelshift_l(X[7], X[8], 16), X[15]);
  const uint32_t t16 = subc_cc(__funnelshift_l(X[8], X[9], 16), X[16]);
  const uint32_t t17 = subc_cc(__funnelshift_l(X[9], X[10], 16), X[17]);
  const uint32_t borrow = subc(0u, 0u) & 1u;
  // q = (X >> 336) - borrow takes the borrow from its lowest limb alone unless that limb
  // is zero (about 2^-32 of the states, also sent to to_ranlux_full), so D = X + q is a
  // single chain over the shifted limbs of X
  const uint32_t q0 = __funnelshift_l(X[10], X[11], 16);
  if (__builtin_expect((t15 & t16 & t17) == 0xFFFFFFFFu || (t15 | t16 | t17) == 0u || q0 < borrow, 0)) {
    to_ranlux_full(X, D);
    return;
  }
  D[0] = add_cc(X[0], q0 - borrow);
#pragma unroll
  for (int k = 1; k < 7; ++k) D[k] = addc_cc(X[k], __funnelshift_l(X[10 + k], X[11 + k], 16));
  D[7] = addc_cc(X[7], X[17] >> 16);
  const uint32_t c8 = addc(0u, 0u);
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) D[k] = X[k];
  // q < 2^240, so a carry out of limb 7 needs limbs 0..7 of X within q of 2^256
  // (about 2^-16 of the states): only then does the chain go on
  if (__builtin_expect(c8 != 0u, 0)) {
    D[8] = add_cc(X[8], 1u);
#pragma unroll
    for (int k = 9; k < kLimbs - 1; ++k) D[k] = addc_cc(X[k], 0u);
    D[kLimbs - 1] = addc(X[kLimbs - 1], 0u);
  }
}

// (D, c) -> X = D - floor(D / 2^336) + c, 336 = 24 (r - s) bits (inverse of to_ranlux).
__device__ __forceinline__ void to_lcg(const uint32_t D[kLimbs], uint32_t c, uint32_t X[kLimbs]) {
  uint32_t Q[8];  // D >> 336: 240 bits
#pragma unroll
  for (int k = 0; k < 7; ++k) Q[k] = shr_pair(D[10 + k], D[11 + k], 16);
  Q[7] = D[17] >> 16;
  X[0] = sub_cc(D[0], Q[0]);
#pragma unroll
  for (int k = 1; k < 8; ++k) X[k] = subc_cc(D[k], Q[k]);
#pragma unroll
  for (int k = 8; k < kLimbs - 1; ++k) X[k] = subc_cc(D[k], 0u);
  X[kLimbs - 1] = subc(D[kLimbs - 1], 0u);
  X[0] = add_cc(X[0], c);
#pragma unroll
  for (int k = 1; k < kLimbs - 1; ++k) X[k] = addc_cc(X[k], 0u);
  X[kLimbs - 1] = addc(X[kLimbs - 1], 0u);
}

// Borrow bit of the RANLUX state: c = X - D + floor(D / 2^336), known to be 0 or 1, so
// the low 32 bits of each term suffice.
__device__ __forceinline__ uint32_t carry_of(const uint32_t X[kLimbs], const uint32_t D[kLimbs]) {
  return X[0] - D[0] + shr_pair(D[10], D[11], 16);
}

// ---------------------------------------------------------------------------------
// Sec. 2.3 outputs.  Word k of the block (k = 0 the oldest) is bits 24k..24k+23 of D;
// the 48-bit value j is bits 48j..48j+47 = word 2j + 2^24 word 2j+1.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t word24(const uint32_t D[kLimbs], int k) {
  const int bit = 24 * k;
  const int limb = bit >> 5, off = bit & 31;
  uint32_t v = D[limb] >> off;
  if (off > 8) v |= D[limb + 1] << (32 - off);
  return v & 0xFFFFFFu;
}

__device__ __forceinline__ uint64_t bits48(const uint32_t D[kLimbs], int j) {
  const int limb = (3 * j) >> 1;  // 48 j / 32
  if ((j & 1) == 0) return ((uint64_t)(D[limb + 1] & 0xFFFFu) << 32) | D[limb];
  return ((uint64_t)(D[limb + 1]) << 16) | (D[limb] >> 16);
}

// 48-bit integer v -> the double v 2^-48 in [0, 1), built with integer operations only
// (the GPU's FP64 pipe is narrow; the conversion is exact because v < 2^53).  The
// leading one of v is moved to bit 52 and the exponent field is set so that the value
// reads v 2^-48: with lz leading zeros in the 64-bit v, the shift is s = lz - 11 and
// the biased exponent 1038 - lz (the leading one itself adds 1 to the field when
// (1026 - s) << 52 is added).  v = 0 maps to +0.0.
__device__ __forceinline__ uint64_t f64_bits_from48_small(uint64_t v) {  // v < 2^32
  const int lz = __clzll((long long)v);  // 32..64
  const int s = lz - 11;
  const uint64_t mant = v << (s & 63);
  const uint64_t bits = mant + ((uint64_t)(1026 - s) << 52);
  return v ? bits : 0ull;
}
__device__ __forceinline__ uint64_t f64_bits_from48_large(uint64_t v) {  // 2^32 <= v < 2^48
  const uint32_t hi = (uint32_t)(v >> 32), lo = (uint32_t)v;
  const uint32_t lz = __clz(hi);  // 16..31, the leading zeros of v as a 64-bit word
  const uint32_t s = lz - 11u;    // 5..20
  const uint32_t mh = __funnelshift_l(lo, hi, s);
  const uint32_t ml = lo << s;
  return ((uint64_t)(mh + ((1037u - lz) << 20)) << 32) | ml;
}
__device__ __forceinline__ uint64_t f64_bits_from48(uint64_t v) {
  return (v >> 32) != 0u ? f64_bits_from48_large(v) : f64_bits_from48_small(v);
}
__device__ __forceinline__ uint32_t bfind_u32(uint32_t x) {  // position of the leading one
  uint32_t p;
  asm("bfind.u32 %0, %1;" : "=r"(p) : "r"(x));
  return p;
}

// The 12 doubles of a block (Sec. 2.3 draw rule, integer construction as in
// f64_bits_from48).  Value j is lo_j + hi_j 2^32 with hi_j < 2^16; when every hi_j is
// nonzero (all but a 12 2^-16 share of the blocks, decided by one OR of the bfind
// results, which are 0xFFFFFFFF for a zero hi_j) the leading
// one of v_j is bit 32 + p_j, p_j = bfind(hi_j): the mantissa is v_j shifted left by
// 20 - p_j and the exponent field (1006 + p_j) + 1 (the leading one adds the 1).
__device__ __forceinline__ void block_f64(const uint32_t D[kLimbs], uint4 v[6]) {
  uint32_t lo[kDoubles], hi[kDoubles];
#pragma unroll
  for (int q = 0; q < 6; ++q) {  // doubles 2q, 2q + 1 = limbs 3q .. 3q + 2
    lo[2 * q] = D[3 * q];
    hi[2 * q] = D[3 * q + 1] & 0xFFFFu;
    lo[2 * q + 1] = __funnelshift_l(D[3 * q + 1], D[3 * q + 2], 16);
    hi[2 * q + 1] = D[3 * q + 2] >> 16;
  }
  uint32_t pos[kDoubles], any = 0;
#pragma unroll
  for (int j = 0; j < kDoubles; ++j) {
    pos[j] = bfind_u32(hi[j]);
    any |= pos[j];
  }
  if (__builtin_expect((int32_t)any >= 0, 1)) {
    uint32_t bh[kDoubles], bl[kDoubles];
#pragma unroll
    for (int j = 0; j < kDoubles; ++j) {
      const uint32_t p = pos[j];  // 0..15
      const uint32_t sh = 20u - p;          // 5..20
      bl[j] = lo[j] << sh;
      bh[j] = __funnelshift_l(lo[j], hi[j], sh) + ((1006u + p) << 20);
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = make_uint4(bl[2 * q], bh[2 * q], bl[2 * q + 1], bh[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const uint64_t a = f64_bits_from48(((uint64_t)hi[2 * q] << 32) | lo[2 * q]);
      const uint64_t b = f64_bits_from48(((uint64_t)hi[2 * q + 1] << 32) | lo[2 * q + 1]);
      v[q] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
    }
  }
}

// The same value with the v < 2^32 case (a 2^-16 share of the values) in a call, so that
// the common case carries no inline copy of it; for kernels with registers to spare.
static __device__ __noinline__ uint64_t f64_bits_from48_small_call(uint64_t v) {
  return f64_bits_from48_small(v);
}
__device__ __forceinline__ uint64_t f64_bits_from48_outlined(uint64_t v) {
  if (__builtin_expect((v >> 32) == 0u, 0)) return f64_bits_from48_small_call(v);
  return f64_bits_from48_large(v);
}

// 24-bit number w -> the binary32 w 2^-24 in [0, 1) (exact), by integer operations:
// the leading one goes to bit 23 and the exponent field makes the value read w 2^-24.
__device__ __forceinline__ uint32_t f32_bits_from24(uint32_t w) {
  const uint32_t lz = __clz(w);  // 8..32
  const uint32_t bits = (w << ((lz - 8u) & 31u)) + ((133u - lz) << 23);
  return w ? bits : 0u;
}

}  // namespace rlxpp
