// Device helpers shared by the kernels that touch the resident state or the power
// table: general modular product, table and state loads/stores, the sticky status,
// and the fixed-window exponentiation of Sec. 2.4 (X <- X A^e, one table product per
// non-zero 4-bit digit of e).
#pragma once
#include "rlxpp_arith.cuh"
#include "rlxpp_internal.h"

namespace rlxpp {

__device__ __forceinline__ void mul_mod(const uint32_t x[kLimbs], const uint32_t y[kLimbs],
                                        uint32_t r[kLimbs]) {
  uint32_t p[2 * kLimbs];
  multiply9x9([&](int i) { return y[i]; }, x, p);
  mod_m(p, r);
}

__device__ __forceinline__ void load18(const uint32_t* __restrict__ src, uint32_t v[kLimbs]) {
  const uint2* s2 = reinterpret_cast<const uint2*>(src);  // entries are 8-byte aligned
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint2 t = __ldg(s2 + k);
    v[2 * k] = t.x;
    v[2 * k + 1] = t.y;
  }
}
__device__ __forceinline__ void store18(uint32_t* dst, const uint32_t v[kLimbs]) {
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) dst[k] = v[k];
}

__device__ __forceinline__ void load_state_D(const StateView& s, uint64_t i, uint32_t D[kLimbs]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint64_t v = s.D[(uint64_t)k * s.stride + i];
    D[2 * k] = (uint32_t)v;
    D[2 * k + 1] = (uint32_t)(v >> 32);
  }
}
__device__ __forceinline__ void store_state_D(const StateView& s, uint64_t i, const uint32_t D[kLimbs]) {
#pragma unroll
  for (int k = 0; k < 9; ++k)
    s.D[(uint64_t)k * s.stride + i] = ((uint64_t)D[2 * k + 1] << 32) | D[2 * k];
}

__device__ __forceinline__ void set_status(int* status, int code) {
  atomicCAS(status, 0, code);
}

// X <- X * prod_w T[w0 + w][digit_w(e)], digits of a 64-bit exponent chunk e; `have`
// tracks whether X holds a value yet (X = 1 otherwise, which is never materialised).
__device__ __forceinline__ void apply_digits(const uint32_t* __restrict__ T, int w0, uint64_t e,
                                             uint32_t X[kLimbs], bool& have) {
#pragma unroll 1
  for (int w = 0; w < 16; ++w) {
    const uint32_t d = (uint32_t)(e >> (4 * w)) & 15u;
    if (d == 0) continue;
    const uint32_t* entry = T + ((size_t)(w0 + w) * kDigits + d) * kLimbs;
    if (!have) {
      load18(entry, X);
      have = true;
    } else {
      uint32_t Y[kLimbs], R[kLimbs];
      load18(entry, Y);
      mul_mod(X, Y, R);
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) X[k] = R[k];
    }
  }
}

}  // namespace rlxpp
