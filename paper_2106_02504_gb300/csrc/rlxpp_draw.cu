// Draw kernels: the refill loop of every stream (Sec. 2: RANLUX numbers -> LCG state,
// multiply9x9 with the luxury multiplier, mod_m, back to RANLUX numbers) fused with the
// output of 24-bit integers, 48-bit doubles (Sec. 2.3) or the sum/histogram consumer of
// the GPU throughput benchmark (Sec. 4.2).
//
// One thread owns one stream and keeps its 576-bit LCG state in registers for the
// whole call.  Every stream of a warp refills at the same step whenever the streams
// start at the same read position and draw the same count (the case the paper's
// staggered-refill experiment in Sec. 4.2 shows to matter), because each refill
// happens at a block boundary and the head of a partly read block is emitted first.
#include "rlxpp_arith.cuh"
#include "rlxpp_internal.h"

// Resident 128-thread blocks per SM the single-level draw kernels are compiled for
// (caps their registers at 65536 / (128 * blocks)).
#ifndef RLXPP_DRAW_MIN_BLOCKS
#define RLXPP_DRAW_MIN_BLOCKS 6
#endif

namespace rlxpp {
namespace {

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
  uint64_t b[kDoubles];
#pragma unroll
  for (int j = 0; j < kDoubles; ++j) b[j] = f64_bits_from48(bits48(D, j));
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

template <int Kind, bool Uniform>
__global__ void __launch_bounds__(kDrawBlock, Uniform ? RLXPP_DRAW_MIN_BLOCKS : 4) k_draw(const DrawArgs a) {
  constexpr int kWarps = kDrawBlock / 32;
  __shared__ unsigned int hist_s[Kind == kDrawSumHist ? kWarps * 256 : 1];
  if (Kind == kDrawSumHist) {
    for (int t = threadIdx.x; t < kWarps * 256; t += kDrawBlock) hist_s[t] = 0;
    __syncthreads();
  }
  const StateView& s = a.s;
  const uint64_t i = (uint64_t)blockIdx.x * kDrawBlock + threadIdx.x;
  if (i < s.n) {
    int64_t cnt, base;
    if (a.counts) {
      cnt = a.counts[i];
      base = a.offsets[i];
    } else {
      cnt = a.count_each;
      base = (int64_t)i * a.count_each;
    }
    const uint32_t meta = s.meta[i];
    uint32_t pos = meta_pos(meta), c = meta_carry(meta);
    const uint32_t lvl = meta_level(meta);
    uint32_t D[kLimbs];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint64_t v = s.D[(uint64_t)k * s.stride + i];
      D[2 * k] = (uint32_t)v;
      D[2 * k + 1] = (uint32_t)(v >> 32);
    }
    uint32_t Areg[kLimbs];
    if (!Uniform) {
      const uint2* src = reinterpret_cast<const uint2*>(s.lux + (size_t)lvl * kLimbs);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const uint2 t = __ldg(src + k);
        Areg[2 * k] = t.x;
        Areg[2 * k + 1] = t.y;
      }
    }
    uint32_t ASreg[9], careg = 0;
    if (!Uniform) {  // half sum of A for the Karatsuba product
      ASreg[0] = add_cc(Areg[0], Areg[9]);
#pragma unroll
      for (int k = 1; k < 9; ++k) ASreg[k] = addc_cc(Areg[k], Areg[9 + k]);
      careg = addc(0u, 0u);
    }
    auto A = [&](int k) { return Uniform ? a.A.a[k] : Areg[k]; };
    auto AS = [&](int k) { return Uniform ? a.A.as[k] : ASreg[k]; };
    const uint32_t ca = Uniform ? a.A.ca : careg;

    Consumer<Kind> out;
    if constexpr (Kind == kDrawU24) out.out = static_cast<uint32_t*>(a.out);
    if constexpr (Kind == kDrawF64) out.out = static_cast<uint64_t*>(a.out);
    if constexpr (Kind == kDrawSumHist) {
      out.sum = 0;
      out.hist = hist_s + (threadIdx.x / 32) * 256;
    }
    constexpr int need = Kind == kDrawU24 ? 1 : 2;  // RANLUX numbers per value
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
    // refills
    if (k < cnt) {
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
#pragma unroll
      for (int q = 0; q < 9; ++q) s.D[(uint64_t)q * s.stride + i] = ((uint64_t)D[2 * q + 1] << 32) | D[2 * q];
    }
    s.meta[i] = meta_pack(pos, c, lvl);
    if constexpr (Kind == kDrawSumHist) {
      uint64_t* sums = static_cast<uint64_t*>(a.out);
      if (sums) sums[i] = a.accumulate_sums ? sums[i] + out.sum : out.sum;
    }
  }
  if (Kind == kDrawSumHist) {
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += kDrawBlock) {
      unsigned long long tot = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) tot += hist_s[w * 256 + t];
      if (tot) atomicAdd(a.hist + t, tot);
    }
  }
}

template <int Kind>
cudaError_t launch_kind(const DrawArgs& a, cudaStream_t st) {
  const unsigned grid = (unsigned)((a.s.n + kDrawBlock - 1) / kDrawBlock);
  if (a.uniform)
    k_draw<Kind, true><<<grid, kDrawBlock, 0, st>>>(a);
  else
    k_draw<Kind, false><<<grid, kDrawBlock, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_draw(int kind, const DrawArgs& a, cudaStream_t st) {
  if (a.s.n == 0) return cudaSuccess;
  switch (kind) {
    case kDrawU24: return launch_kind<kDrawU24>(a, st);
    case kDrawF64: return launch_kind<kDrawF64>(a, st);
    case kDrawSumHist: return launch_kind<kDrawSumHist>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rlxpp
