// The per-stream draw loop shared by the draw kernels and the request kernel: emit the
// unread part of the current block, then refill (RANLUX numbers -> LCG state,
// multiply9x9 by A, mod_m, back to RANLUX numbers; Sec. 2) and emit until the count is
// reached, with the value written, stored or consumed by a Consumer.
#pragma once
#include "rlxpp_arith.cuh"
#include "rlxpp_fixmath.cuh"
#include "rlxpp_internal.h"

namespace rlxpp {

// 48 bits starting at RANLUX number w (w + 1 < 24), i.e. bits 24w..24w+47 of D.
__device__ __forceinline__ uint64_t bits48_at_word(const uint32_t D[kLimbs], int w) {
  const int bit = 24 * w;
  const int limb = bit >> 5, off = bit & 31;
  uint64_t v = (uint64_t)D[limb];
  if (limb + 1 < kLimbs) v |= (uint64_t)D[limb + 1] << 32;
  v >>= off;
  if (off > 16 && limb + 2 < kLimbs) v |= (uint64_t)D[limb + 2] << (64 - off);
  return v & 0xFFFFFFFFFFFFull;
}

__device__ __forceinline__ void st_v4_u64(uint64_t* p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
  asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
               : "memory");
}
__device__ __forceinline__ void st_v8_u32(uint32_t* p, const uint32_t* v) {
  asm volatile("st.global.v8.u32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}

// A full block of 12 doubles to o[0..11]; 32-byte vector stores when aligned.
__device__ __forceinline__ void store_block_f64(uint64_t* o, const uint32_t D[kLimbs]) {
  uint4 v[6];
  block_f64(D, v);
  uint64_t b[kDoubles];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    b[2 * q] = ((uint64_t)v[q].y << 32) | v[q].x;
    b[2 * q + 1] = ((uint64_t)v[q].w << 32) | v[q].z;
  }
  const uintptr_t addr = reinterpret_cast<uintptr_t>(o);
  if ((addr & 31) == 0) {
#pragma unroll
    for (int j = 0; j < kDoubles; j += 4) st_v4_u64(o + j, b[j], b[j + 1], b[j + 2], b[j + 3]);
  } else if ((addr & 15) == 0) {
#pragma unroll
    for (int j = 0; j < kDoubles; j += 2)
      *reinterpret_cast<ulonglong2*>(o + j) = make_ulonglong2(b[j], b[j + 1]);
  } else {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j) o[j] = b[j];
  }
}

// A full block of 24 numbers to o[0..23].
__device__ __forceinline__ void store_block_u24(uint32_t* o, const uint32_t D[kLimbs]) {
  uint32_t w[kWords];
#pragma unroll
  for (int j = 0; j < kWords; ++j) w[j] = word24(D, j);
  const uintptr_t addr = reinterpret_cast<uintptr_t>(o);
  if ((addr & 31) == 0) {
#pragma unroll
    for (int j = 0; j < kWords; j += 8) st_v8_u32(o + j, w + j);
  } else if ((addr & 15) == 0) {
#pragma unroll
    for (int j = 0; j < kWords; j += 4)
      *reinterpret_cast<uint4*>(o + j) = make_uint4(w[j], w[j + 1], w[j + 2], w[j + 3]);
  } else {
#pragma unroll
    for (int j = 0; j < kWords; ++j) o[j] = w[j];
  }
}

template <int Kind>
struct Consumer;

template <>
struct Consumer<kDrawU24> {
  uint32_t* out;
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t idx) {
    out[idx] = word24(D, w);
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t idx) {
    store_block_u24(out + idx, D);
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t idx, int64_t n) {
#pragma unroll
    for (int j = 0; j < kWords; ++j)
      if (j < n) out[idx + j] = word24(D, j);
  }
};

template <>
struct Consumer<kDrawF32> {
  uint32_t* out;
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t idx) {
    out[idx] = f32_bits_from24(word24(D, w));
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t idx) {
    uint32_t* o = out + idx;
    uint32_t w[kWords];
#pragma unroll
    for (int j = 0; j < kWords; ++j) w[j] = f32_bits_from24(word24(D, j));
    if ((reinterpret_cast<uintptr_t>(o) & 15) == 0) {
#pragma unroll
      for (int j = 0; j < kWords; j += 4)
        *reinterpret_cast<uint4*>(o + j) = make_uint4(w[j], w[j + 1], w[j + 2], w[j + 3]);
    } else {
#pragma unroll
      for (int j = 0; j < kWords; ++j) o[j] = w[j];
    }
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t idx, int64_t n) {
#pragma unroll
    for (int j = 0; j < kWords; ++j)
      if (j < n) out[idx + j] = f32_bits_from24(word24(D, j));
  }
};

template <>
struct Consumer<kDrawF64> {
  uint64_t* out;
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t idx) {
    out[idx] = f64_bits_from48(bits48_at_word(D, w));
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t idx) {
    store_block_f64(out + idx, D);
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t idx, int64_t n) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j)
      if (j < n) out[idx + j] = f64_bits_from48(bits48(D, j));
  }
};

// Exact sum of the 48-bit integers and a per-warp 256-bin histogram of their top 8 bits.
template <>
struct Consumer<kDrawSumHist> {
  uint64_t sum;
  unsigned int* hist;  // this warp's 256 shared-memory bins
  __device__ __forceinline__ void take(uint64_t v) {
    sum += v;
    atomicAdd(hist + (unsigned)(v >> 40), 1u);
  }
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t) {
    take(bits48_at_word(D, w));
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j) take(bits48(D, j));
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t, int64_t n) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j)
      if (j < n) take(bits48(D, j));
  }
};

// Gaussian doubles by the Box-Muller transform (Box and Muller, Ann. Math. Statist. 29,
// 1958) on consecutive pairs (d_a, d_b) of the stream's doubles: u1 = 1 - d_a in (0, 1]
// (exact: (2^48 - v_a) 2^-48), r = sqrt(-2 ln u1), z_a = r cos(2 pi d_b),
// z_b = r sin(2 pi d_b).  The draw loop feeds it 2 ceil(n / 2) doubles, value j at
// output index base + j; pairs start at even j; an index at or past `end` (the last
// sine of an odd count) is not written.  ln, sqrt, cos and sin are the integer-pipe
// routines of rlxpp_fixmath.cuh, applied to the 48-bit integers themselves.
template <>
struct Consumer<kDrawNormal> {
  double* out;
  int64_t base, end;
  uint64_t va;  // first value of the current pair, as its 48-bit integer
  __device__ __forceinline__ void take(uint64_t v, int64_t idx) {
    if (((idx - base) & 1) == 0) {
      va = v;
      return;
    }
    double z0, z1;
    fx_box_muller48(va, v, z0, z1);
    out[idx - 1] = z0;
    if (idx < end) out[idx] = z1;
  }
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t idx) {
    take(bits48_at_word(D, w), idx);
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t idx) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j) take(bits48(D, j), idx + j);
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t idx, int64_t n) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j)
      if (j < n) take(bits48(D, j), idx + j);
  }
};

// Exponential doubles (rate 1) by inversion: x = -ln(1 - d) for each double d of the
// stream (1 - d = (2^48 - v) 2^-48 exactly, in (0, 1]; d = 0 gives +0), with the
// integer-pipe logarithm of rlxpp_fixmath.cuh.
__device__ __forceinline__ double exp_from48(uint64_t v) { return fx_exponential48(v); }
template <>
struct Consumer<kDrawExp> {
  double* out;
  __device__ __forceinline__ void value_at_word(const uint32_t D[kLimbs], int w, int64_t idx) {
    out[idx] = exp_from48(bits48_at_word(D, w));
  }
  __device__ __forceinline__ void block(const uint32_t D[kLimbs], int64_t idx) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j) out[idx + j] = exp_from48(bits48(D, j));
  }
  __device__ __forceinline__ void partial(const uint32_t D[kLimbs], int64_t idx, int64_t n) {
#pragma unroll
    for (int j = 0; j < kDoubles; ++j)
      if (j < n) out[idx + j] = exp_from48(bits48(D, j));
  }
};

// Draws cnt values for one stream.  On entry D holds the RANLUX numbers of the current
// block, c its borrow and pos the numbers already read; values go to out at indices
// base, base + 1, ...  On return D, c and pos describe the stream after the draw.
// Returns true when at least one refill happened (then D and c changed).
template <int Kind, class AFn, class ASFn>
__device__ __forceinline__ bool draw_stream(Consumer<Kind>& out, uint32_t D[kLimbs], uint32_t& c, uint32_t& pos,
                                            AFn A, ASFn AS, uint32_t ca, int64_t cnt, int64_t base) {
  constexpr int need = (Kind == kDrawU24 || Kind == kDrawF32) ? 1 : 2;  // RANLUX numbers per value
  constexpr int per_block = kWords / need;
  int64_t k = 0;
  // head: the unread part of the current block
  if (cnt > 0 && pos + need <= (uint32_t)kWords) {
    const int64_t room = (kWords - pos) / need;
    const int64_t h = cnt < room ? cnt : room;
#pragma unroll
    for (int w = 0; w + need <= kWords; ++w) {
      const int d = w - (int)pos;
      if (d >= 0 && d % need == 0 && d / need < h) out.value_at_word(D, w, base + d / need);
    }
    k = h;
    pos += (uint32_t)(h * need);
  }
  if (k >= cnt) return false;
  // refills
  uint32_t X[kLimbs];
  to_lcg(D, c, X);
#pragma unroll 1
  while (true) {
    uint32_t P[2 * kLimbs];
    multiply9x9_split(A, AS, ca, X, P);
    mod_m(P, X);
    to_ranlux(X, D);
    const int64_t rem = cnt - k;
    if (rem >= per_block) {
      out.block(D, base + k);
      k += per_block;
      pos = kWords;
      if (k == cnt) break;
    } else {
      out.partial(D, base + k, rem);
      k = cnt;
      pos = (uint32_t)(rem * need);
      break;
    }
  }
  c = carry_of(X, D);
  return true;
}

}  // namespace rlxpp
