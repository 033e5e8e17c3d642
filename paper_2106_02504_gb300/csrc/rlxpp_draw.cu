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
#include "rlxpp_drawloop.cuh"
#include "rlxpp_internal.h"

// Resident 128-thread blocks per SM the single-level draw kernels are compiled for
// (caps their registers at 65536 / (128 * blocks)).
#ifndef RLXPP_DRAW_MIN_BLOCKS
#define RLXPP_DRAW_MIN_BLOCKS 6
#endif

namespace rlxpp {
namespace {

template <int Kind, bool Uniform>
__global__ void __launch_bounds__(kDrawBlock, (Uniform && Kind != kDrawNormal && Kind != kDrawExp) ? RLXPP_DRAW_MIN_BLOCKS : 4) k_draw(const DrawArgs a) {
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
    if constexpr (Kind == kDrawF32) out.out = static_cast<uint32_t*>(a.out);
    if constexpr (Kind == kDrawSumHist) {
      out.sum = 0;
      out.hist = hist_s + (threadIdx.x / 32) * 256;
    }
    if constexpr (Kind == kDrawExp) out.out = static_cast<double*>(a.out);
    if constexpr (Kind == kDrawNormal) {  // n normals take 2 ceil(n / 2) doubles
      out.out = static_cast<double*>(a.out);
      out.base = base;
      out.end = base + cnt;
      out.va = 0;
      cnt += cnt & 1;
    }
    if (draw_stream<Kind>(out, D, c, pos, A, AS, ca, cnt, base)) {
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

// Raw LCG doubles (Sec. 2.3's biased form, for comparison): the 52 bits of the LCG state
// X starting at bit 52 k (k <= 10, so the two limbs from bit 52 k's limb on exist), and
// v 2^-52 as a double built with integer operations (exact: v < 2^52): the leading one
// moves to bit 52, where it adds one to the exponent field 1033 - lz placed above it.
__device__ __forceinline__ uint64_t bits52(const uint32_t X[kLimbs], int k) {
  const int bit = 52 * k, limb = bit >> 5, off = bit & 31;
  uint64_t v = ((uint64_t)X[limb] | ((uint64_t)X[limb + 1] << 32)) >> off;
  if (off > 12 && limb + 2 < kLimbs) v |= (uint64_t)X[limb + 2] << (64 - off);
  return v & ((1ull << 52) - 1);
}
__device__ __forceinline__ uint64_t f64_bits_from52(uint64_t v) {
  if (v == 0) return 0;
  const int lz = __clzll((long long)v);  // 12 .. 63
  return (v << (lz - 11)) + ((uint64_t)(1033 - lz) << 52);
}

// Raw LCG doubles: each stream starts with a refill and emits 11 values of every new
// LCG state until its count is reached; the stream is left at the end of its last
// block (read position 24).
template <bool Uniform>
__global__ void __launch_bounds__(kDrawBlock, 4) k_draw_raw(const DrawArgs a) {
  const StateView& s = a.s;
  const uint64_t i = (uint64_t)blockIdx.x * kDrawBlock + threadIdx.x;
  if (i >= s.n) return;
  int64_t cnt, base;
  if (a.counts) {
    cnt = a.counts[i];
    base = a.offsets[i];
  } else {
    cnt = a.count_each;
    base = (int64_t)i * a.count_each;
  }
  if (cnt <= 0) return;
  const uint32_t meta = s.meta[i];
  uint32_t c = meta_carry(meta);
  const uint32_t lvl = meta_level(meta);
  uint32_t D[kLimbs];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint64_t v = s.D[(uint64_t)k * s.stride + i];
    D[2 * k] = (uint32_t)v;
    D[2 * k + 1] = (uint32_t)(v >> 32);
  }
  uint32_t Areg[kLimbs], ASreg[9], careg = 0;
  if (!Uniform) {
    const uint2* src = reinterpret_cast<const uint2*>(s.lux + (size_t)lvl * kLimbs);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const uint2 t = __ldg(src + k);
      Areg[2 * k] = t.x;
      Areg[2 * k + 1] = t.y;
    }
    ASreg[0] = add_cc(Areg[0], Areg[9]);
#pragma unroll
    for (int k = 1; k < 9; ++k) ASreg[k] = addc_cc(Areg[k], Areg[9 + k]);
    careg = addc(0u, 0u);
  }
  auto A = [&](int k) { return Uniform ? a.A.a[k] : Areg[k]; };
  auto AS = [&](int k) { return Uniform ? a.A.as[k] : ASreg[k]; };
  const uint32_t ca = Uniform ? a.A.ca : careg;
  uint64_t* out = static_cast<uint64_t*>(a.out) + base;
  uint32_t X[kLimbs];
  to_lcg(D, c, X);
#pragma unroll 1
  for (int64_t k0 = 0; k0 < cnt; k0 += 11) {
    uint32_t P[2 * kLimbs];
    multiply9x9_split(A, AS, ca, X, P);
    mod_m(P, X);
#pragma unroll
    for (int k = 0; k < 11; ++k)
      if (k0 + k < cnt) out[k0 + k] = f64_bits_from52(bits52(X, k));
  }
  to_ranlux(X, D);
  c = carry_of(X, D);
#pragma unroll
  for (int q = 0; q < 9; ++q) s.D[(uint64_t)q * s.stride + i] = ((uint64_t)D[2 * q + 1] << 32) | D[2 * q];
  s.meta[i] = meta_pack((uint32_t)kWords, c, lvl);
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
    case kDrawF32: return launch_kind<kDrawF32>(a, st);
    case kDrawNormal: return launch_kind<kDrawNormal>(a, st);
    case kDrawExp: return launch_kind<kDrawExp>(a, st);
    case kDrawRaw52: {
      const unsigned grid = (unsigned)((a.s.n + kDrawBlock - 1) / kDrawBlock);
      if (a.uniform)
        k_draw_raw<true><<<grid, kDrawBlock, 0, st>>>(a);
      else
        k_draw_raw<false><<<grid, kDrawBlock, 0, st>>>(a);
      return cudaGetLastError();
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace rlxpp
