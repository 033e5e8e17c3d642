// Warp-cooperative refill: one warp per stream, for draws from few streams, where one
// thread per stream leaves the GPU idle and the refill's latency is what counts (a
// single stream read in order).  Lane l holds 32-bit limb l of the 576-bit numbers;
// the steps are those of Sec. 2: RANLUX numbers -> LCG state, multiply9x9 (Sec. 2.1),
// mod_m (Sec. 2.2), back to RANLUX numbers (Sec. 2.3), then the output.
//
// Every multi-limb addition resolves its carries in one step across the warp: each lane
// adds its limbs, the lanes whose sum overflowed (generate) and whose sum is all ones
// (propagate) are collected by ballots, and the carries into the lanes are
// ((G << 1) + P) ^ P — a carry enters lane l exactly when some lane below generated one
// and every lane in between propagates it.  Subtractions do the same with borrows.
#include "rlxpp_arith.cuh"
#include "rlxpp_batch.h"
#include "rlxpp_drawloop.cuh"
#include "rlxpp_internal.h"
#include "rlxpp_state.cuh"

namespace rlxpp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarpBlock = 128;  // threads per block: 4 streams
constexpr int kWarpsPerBlock = kWarpBlock / 32;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// x + y over the 32 lanes; *cout (if given) gets the carry out of lane 31.
__device__ __forceinline__ uint32_t wadd(uint32_t x, uint32_t y, uint32_t* cout = nullptr) {
  const uint32_t s = x + y;
  const uint32_t g = __ballot_sync(kFull, s < x);
  const uint32_t p = __ballot_sync(kFull, s == 0xFFFFFFFFu);
  const uint64_t c = (((uint64_t)g << 1) + p) ^ p;
  if (cout) *cout = (uint32_t)(c >> 32) & 1u;
  return s + (uint32_t)((c >> lane_id()) & 1u);
}

// x - y over the 32 lanes; *bout (if given) gets the borrow out of lane 31.
__device__ __forceinline__ uint32_t wsub(uint32_t x, uint32_t y, uint32_t* bout = nullptr) {
  const uint32_t d = x - y;
  const uint32_t g = __ballot_sync(kFull, x < y);
  const uint32_t p = __ballot_sync(kFull, d == 0u);
  const uint64_t c = (((uint64_t)g << 1) + p) ^ p;
  if (bout) *bout = (uint32_t)(c >> 32) & 1u;
  return d - (uint32_t)((c >> lane_id()) & 1u);
}

// Limbs from per-lane sums v_l < 2^35 (the number sum_l v_l 2^(32 l)): the high part of
// each lane goes to the next lane in one step, which leaves carries of at most 1, then
// one lookahead resolves them; the part past lane 31 is dropped.
__device__ __forceinline__ uint32_t wsettle(uint64_t v) {
  const uint32_t lo = (uint32_t)v, hi = (uint32_t)(v >> 32);
  const uint32_t hin = __shfl_up_sync(kFull, hi, 1);
  const uint64_t u = (uint64_t)lo + (lane_id() ? hin : 0u);  // < 2^32 + 2^3
  const uint32_t r = (uint32_t)u;
  const uint32_t g = __ballot_sync(kFull, (u >> 32) != 0);
  const uint32_t p = __ballot_sync(kFull, r == 0xFFFFFFFFu);
  const uint64_t c = (((uint64_t)g << 1) + p) ^ p;
  return r + (uint32_t)((c >> lane_id()) & 1u);
}

// lane l <- y of lane l - k (0 for l < k), and of lane l + k (0 past lane 31)
__device__ __forceinline__ uint32_t wup(uint32_t y, int k) {
  const uint32_t v = __shfl_up_sync(kFull, y, k);
  return lane_id() >= (unsigned)k ? v : 0u;
}
__device__ __forceinline__ uint32_t wdown(uint32_t y, int k) {
  const uint32_t v = __shfl_down_sync(kFull, y, k);
  return lane_id() + (unsigned)k < 32u ? v : 0u;
}

// y << 240 (7 limbs and 16 bits) and y >> 336 (10 limbs and 16 bits)
__device__ __forceinline__ uint32_t wshl240(uint32_t y) { return __funnelshift_l(wup(y, 8), wup(y, 7), 16); }
__device__ __forceinline__ uint32_t wshr336(uint32_t y) { return __funnelshift_r(wdown(y, 10), wdown(y, 11), 16); }

// Entries of a 36-limb number kept as two halves per lane (entries l and 18 + l on
// lanes 0..17): the entry k below, as (a', b') for the halves (a, b).
__device__ __forceinline__ void wprev(uint32_t a, uint32_t b, int k, uint32_t& pa, uint32_t& pb) {
  const unsigned l = lane_id();
  const int src = (int)((l + 18u - (unsigned)k) % 18u);
  const uint32_t va = __shfl_sync(kFull, a, src);
  const uint32_t vb = __shfl_sync(kFull, b, src);
  pa = l >= (unsigned)k ? va : 0u;
  pb = l >= (unsigned)k ? vb : va;
}

// (a, b) += (xa, xb) over the 36 entries (no carry out of entry 35 by the caller's bounds).
__device__ __forceinline__ void wadd36(uint32_t& a, uint32_t& b, uint32_t xa, uint32_t xb) {
  const unsigned l = lane_id();
  const bool in = l < 18;  // lanes 18..31 hold no entries
  const uint32_t sa = a + xa, sb = b + xb;
  const uint64_t G =
      (uint64_t)__ballot_sync(kFull, in && sa < a) | ((uint64_t)__ballot_sync(kFull, in && sb < b) << 18);
  const uint64_t P = (uint64_t)__ballot_sync(kFull, in && sa == 0xFFFFFFFFu) |
                     ((uint64_t)__ballot_sync(kFull, in && sb == 0xFFFFFFFFu) << 18);
  const uint64_t C = ((G << 1) + P) ^ P;
  a = l < 18 ? sa + (uint32_t)((C >> l) & 1u) : 0u;
  b = l < 18 ? sb + (uint32_t)((C >> (l + 18)) & 1u) : 0u;
}

// P = A X (Sec. 2.1).  Lane l < 18 forms the column sums of entries l and 18 + l
// (sum_{i <= l} A_i X_{l-i} and sum_{i > l} A_i X_{l+18-i}: 18 products together), as
// sums of the products' low and high halves, then the 36 limbs follow by one carry step.
// Out: L = limbs 0..17, H = limbs 18..35 (lanes 0..17; other lanes 0).
template <class AFn>
__device__ __forceinline__ void wmul(AFn A, uint32_t X, uint32_t& L, uint32_t& H) {
  const unsigned l = lane_id();
  uint64_t loA = 0, hiA = 0, loB = 0, hiB = 0;
#pragma unroll
  for (int i = 0; i < 18; ++i) {
    const int src = (int)((l + 18u - (unsigned)i) % 18u);
    const uint32_t x = __shfl_sync(kFull, X, src);
    const uint64_t pr = (uint64_t)A(i) * x;
    const uint32_t plo = (uint32_t)pr, phi = (uint32_t)(pr >> 32);
    if (i <= (int)l) {
      loA += plo;
      hiA += phi;
    } else {
      loB += plo;
      hiB += phi;
    }
  }
  if (l >= 18) loA = hiA = loB = hiB = 0;
  // entry e receives lo32(lo_e) + hi32(lo_{e-1}) + lo32(hi_{e-1}) + hi32(hi_{e-2})
  uint32_t p1a, p1b, p2a, p2b, p3a, p3b;
  wprev((uint32_t)(loA >> 32), (uint32_t)(loB >> 32), 1, p1a, p1b);
  wprev((uint32_t)hiA, (uint32_t)hiB, 1, p2a, p2b);
  wprev((uint32_t)(hiA >> 32), (uint32_t)(hiB >> 32), 2, p3a, p3b);
  const uint64_t wa = (uint64_t)(uint32_t)loA + p1a + p2a + p3a;  // < 2^34
  const uint64_t wb = (uint64_t)(uint32_t)loB + p1b + p2b + p3b;
  uint32_t ca, cb;
  wprev((uint32_t)(wa >> 32), (uint32_t)(wb >> 32), 1, ca, cb);
  L = (uint32_t)wa;
  H = (uint32_t)wb;
  wadd36(L, H, ca, cb);
}

// 2 m limb by lane (m = 2^576 - 2^240 + 1): 2, zeros, 0xFFFE0000 at lane 7, all ones on
// lanes 8..17, 1 at lane 18.
__device__ __forceinline__ uint32_t two_m_limb(unsigned l) {
  return l == 0 ? 2u : (l < 7 ? 0u : (l == 7 ? 0xFFFE0000u : (l < 18 ? 0xFFFFFFFFu : (l == 18 ? 1u : 0u))));
}
// 2^240 - 1 limb by lane
__device__ __forceinline__ uint32_t pow240m1_limb(unsigned l) {
  return l < 7 ? 0xFFFFFFFFu : (l == 7 ? 0xFFFFu : 0u);
}

// P = L + H 2^576 -> P mod m in [0, m) (Sec. 2.2): with 2^576 = 2^240 - 1 (mod m),
// H = H0 + H1 2^336 (H0 < 2^336, H1 < 2^240),
//   P = L - H + H0 2^240 + H1 2^240 - H1 (mod m);
// 2 m is added to keep it positive (below 2^579), the top bits t above 2^576 are folded
// back as t (2^240 - 1), then rarely once more, and the result is reduced below m.
__device__ __forceinline__ uint32_t wmod_m(uint32_t L, uint32_t H) {
  const unsigned l = lane_id();
  const uint32_t H0 = l < 10 ? H : (l == 10 ? (H & 0xFFFFu) : 0u);
  const uint32_t H1 = wshr336(H);  // lanes 0..7
  // A2 = H1 2^240 = (H >> 96) with bits below 240 cleared: limb 7 = the top half of H's
  // limb 10, limbs 8..14 = H's limbs 11..17 (one shuffle by three lanes)
  const uint32_t H3 = wdown(H, 3);
  const uint32_t A1 = wshl240(H0);
  const uint32_t A2 = l == 7 ? (H3 & 0xFFFF0000u) : ((l >= 8 && l < 15) ? H3 : 0u);
  // V = L + A1 + A2 + 2m - H - H1 on 19 lanes (V < 2^579), the subtrahends as their
  // complements: -Y = ~Y + 1 - 2^608 within 19 lanes, so every lane's sum is
  // non-negative and the 2 2^608 that remain fall past lane 18 and are dropped.
  uint64_t v = (uint64_t)L + A1 + A2 + two_m_limb(l) + (uint32_t)~H + (uint32_t)~H1 + (l == 0 ? 2u : 0u);
  if (l >= 19) v = 0;
  uint32_t V = wsettle(v);
  const uint32_t t = __shfl_sync(kFull, V, 18);  // 0..7, almost always nonzero
  if (l >= 18) V = 0;
  {  // + t (2^240 - 1) = (t - 1) 2^240 + (2^240 - t) for t >= 1 (non-negative limbs); 0 for t = 0
    const uint32_t f = l == 0 ? 0u - t : (l < 7 ? 0xFFFFFFFFu : (l == 7 ? (((t - 1u) << 16) | 0xFFFFu) : 0u));
    V = wadd(V, t ? f : 0u);
  }
  if (__shfl_sync(kFull, V, 18)) {  // another 2^576 (rare): + 2^240 - 1
    if (l == 18) V = 0;
    V = wadd(V, pow240m1_limb(l));
  }
  // V >= m needs bits 240..575 all set (rare); then V - m = V + 2^240 - 1 - 2^576
  const bool top_ones = (l >= 8 && l < 18) ? V == 0xFFFFFFFFu : (l == 7 ? (V >> 16) == 0xFFFFu : true);
  if (__all_sync(kFull, top_ones)) {
    const uint32_t E = wadd(V, pow240m1_limb(l));
    if (__shfl_sync(kFull, E, 18)) V = l == 18 ? 0u : E;
  }
  return V;
}

// X -> D = floor(2^576 X / m) (Sec. 2.3): D = X + q, q = (X >> 336) - [S < X] with
// S = (X << 240) mod 2^576, unless T = S - X has limbs 15..17 all ones (about 2^-96 of
// the states), where q may be one more: that case goes through the single-thread
// conversion on lane 0 (scratch: this warp's 36 words of shared memory).
__device__ __forceinline__ uint32_t wto_ranlux(uint32_t X, uint32_t* scratch) {
  const unsigned l = lane_id();
  uint32_t S = wshl240(X);  // every lane shuffles; lanes 18.. then drop their part
  if (l >= 18) S = 0u;
  const uint32_t Q336 = wshr336(X);  // needed below; shuffled early, beside wsub's votes
  uint32_t b;
  const uint32_t T = wsub(S, X, &b);
  const bool top3 = (l >= 15 && l < 18) ? T == 0xFFFFFFFFu : true;
  if (__all_sync(kFull, top3)) {
    if (l < 18) scratch[l] = X;
    __syncwarp();
    if (l == 0) {
      uint32_t Xs[kLimbs], Ds[kLimbs];
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) Xs[k] = scratch[k];
      to_ranlux_full(Xs, Ds);
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) scratch[18 + k] = Ds[k];
    }
    __syncwarp();
    const uint32_t D = l < 18 ? scratch[18 + l] : 0u;
    __syncwarp();
    return D;
  }
  // D = X + (X >> 336) - b = X + (X >> 336) + b (2^576 - 1) mod 2^576 (D < 2^576)
  uint64_t v = (uint64_t)X + Q336 + (b ? 0xFFFFFFFFu : 0u);
  if (l >= 18) v = 0;
  const uint32_t D = wsettle(v);
  return l < 18 ? D : 0u;
}

// (D, c) -> X = D - (D >> 336) + c, and the carry c = X - D + (D >> 336) of a state.
__device__ __forceinline__ uint32_t wto_lcg(uint32_t D, uint32_t c) {
  const uint32_t X = wsub(D, wshr336(D));
  return wadd(X, lane_id() == 0 ? c : 0u);
}
__device__ __forceinline__ uint32_t wcarry(uint32_t X, uint32_t D) {
  const uint32_t v = wadd(wsub(X, D), wshr336(D));
  return __shfl_sync(kFull, v, 0);
}

// The 24-bit number at word w and the 48-bit integer at words w, w + 1 of D.
__device__ __forceinline__ uint32_t wword24(uint32_t D, int w) {
  const int k = (24 * w) >> 5, sh = (24 * w) & 31;
  const uint32_t a = __shfl_sync(kFull, D, k & 31), b = __shfl_sync(kFull, D, (k + 1) & 31);
  return __funnelshift_r(a, b, sh) & 0xFFFFFFu;
}
__device__ __forceinline__ uint64_t wbits48(uint32_t D, int w) {
  const int k = (24 * w) >> 5, sh = (24 * w) & 31;
  const uint32_t a = __shfl_sync(kFull, D, k & 31), b = __shfl_sync(kFull, D, (k + 1) & 31),
                 c = __shfl_sync(kFull, D, (k + 2) & 31);
  return ((uint64_t)(__funnelshift_r(b, c, sh) & 0xFFFFu) << 32) | __funnelshift_r(a, b, sh);
}

template <int Kind, bool Uniform>
__global__ void __launch_bounds__(kWarpBlock) k_draw_warp(const DrawArgs a) {
  __shared__ unsigned int hist_s[Kind == kDrawSumHist ? kWarpsPerBlock * 256 : 1];
  __shared__ uint32_t scratch_s[kWarpsPerBlock][36];
  const unsigned l = lane_id();
  const int warp = threadIdx.x / 32;
  if (Kind == kDrawSumHist) {
    for (int t = threadIdx.x; t < kWarpsPerBlock * 256; t += kWarpBlock) hist_s[t] = 0;
    __syncthreads();
  }
  const StateView& s = a.s;
  const uint64_t i = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;
  uint64_t sum = 0;
  if (i < s.n) {  // the whole warp: one stream
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
    uint32_t D = 0;
    if (l < 18) {
      const uint64_t v = s.D[(uint64_t)(l / 2) * s.stride + i];
      D = (l & 1) ? (uint32_t)(v >> 32) : (uint32_t)v;
    }
    const uint32_t* luxl = s.lux + (size_t)lvl * kLimbs;
    auto A = [&](int k) { return Uniform ? a.A.a[k] : __ldg(luxl + k); };
    constexpr int need = (Kind == kDrawU24 || Kind == kDrawF32) ? 1 : 2;
    constexpr int per_block = kWords / need;
    unsigned int* hist = hist_s + warp * 256;
    // the value of lane j for a block read from word w0 on (u24 / f32: word w0 + j;
    // f64 and the fused consumer: words w0 + 2j, w0 + 2j + 1)
    auto emit = [&](int w0, int64_t idx0, int64_t nvals) {
      const int j = (int)l;
      const int w = w0 + j * need;
      const bool on = j < nvals && w + need <= kWords;
      if constexpr (Kind == kDrawU24 || Kind == kDrawF32) {
        const uint32_t v = wword24(D, w < kWords ? w : 0);
        if (on) {
          if constexpr (Kind == kDrawU24)
            static_cast<uint32_t*>(a.out)[idx0 + j] = v;
          else
            static_cast<uint32_t*>(a.out)[idx0 + j] = f32_bits_from24(v);
        }
      } else {
        const uint64_t v = wbits48(D, w < kWords - 1 ? w : 0);
        if constexpr (Kind == kDrawF64) {
          if (on) static_cast<uint64_t*>(a.out)[idx0 + j] = f64_bits_from48(v);
        } else {  // fused sum and histogram
          if (on) {
            sum += v;
            atomicAdd(hist + (unsigned)(v >> 40), 1u);
          }
        }
      }
    };
    int64_t k = 0;
    if (cnt > 0 && pos + need <= (uint32_t)kWords) {  // head of the current block
      const int64_t room = (kWords - pos) / need;
      const int64_t h = cnt < room ? cnt : room;
      emit((int)pos, base, h);
      k = h;
      pos += (uint32_t)(h * need);
    }
    if (k < cnt) {
      uint32_t X = wto_lcg(D, c);
#pragma unroll 1
      while (true) {
        uint32_t L, H;
        wmul(A, l < 18 ? X : 0u, L, H);
        X = wmod_m(L, H);
        D = wto_ranlux(X, scratch_s[warp]);
        const int64_t rem = cnt - k;
        if (rem >= per_block) {
          emit(0, base + k, per_block);
          k += per_block;
          pos = kWords;
          if (k == cnt) break;
        } else {
          emit(0, base + k, rem);
          k = cnt;
          pos = (uint32_t)(rem * need);
          break;
        }
      }
      c = wcarry(X, D);
      const uint32_t hiD = __shfl_down_sync(kFull, D, 1);
      if (l < 18 && (l & 1) == 0) s.D[(uint64_t)(l / 2) * s.stride + i] = ((uint64_t)hiD << 32) | D;
    }
    if (l == 0) s.meta[i] = meta_pack(pos, c, lvl);
    if constexpr (Kind == kDrawSumHist) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
      uint64_t* sums = static_cast<uint64_t*>(a.out);
      if (l == 0 && sums) sums[i] = a.accumulate_sums ? sums[i] + sum : sum;
    }
  }
  if (Kind == kDrawSumHist) {
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += kWarpBlock) {
      unsigned long long tot = 0;
#pragma unroll
      for (int w = 0; w < kWarpsPerBlock; ++w) tot += hist_s[w * 256 + t];
      if (tot) atomicAdd(a.hist + t, tot);
    }
  }
}

// Unit tests of the warp arithmetic, one warp per item.  op 0: in = 18 uint64 (1152 bits)
// -> out = in mod m (9 uint64); op 1: in = X < m (9 uint64) -> out = D (9 uint64) and
// carry[i].
__global__ void __launch_bounds__(kWarpBlock) k_test_warp(int op, const uint64_t* __restrict__ in,
                                                          uint64_t* __restrict__ out, uint32_t* __restrict__ carry,
                                                          uint64_t n) {
  __shared__ uint32_t scratch_s[kWarpsPerBlock][36];
  const unsigned l = lane_id();
  const int warp = threadIdx.x / 32;
  const uint64_t i = (uint64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (i >= n) return;  // the whole warp
  auto limb = [](const uint64_t* p, unsigned k) {
    return (k & 1) ? (uint32_t)(p[k / 2] >> 32) : (uint32_t)p[k / 2];
  };
  uint32_t r;
  if (op == 0) {
    const uint64_t* p = in + 18 * i;
    const uint32_t L = l < 18 ? limb(p, l) : 0u;
    const uint32_t H = l < 18 ? limb(p, 18 + l) : 0u;
    r = wmod_m(L, H);
  } else {
    const uint64_t* p = in + 9 * i;
    const uint32_t X = l < 18 ? limb(p, l) : 0u;
    r = wto_ranlux(X, scratch_s[warp]);
    const uint32_t c = wcarry(X, r);
    if (l == 0) carry[i] = c;
  }
  const uint32_t hi = __shfl_down_sync(kFull, r, 1);
  if (l < 18 && (l & 1) == 0) out[9 * i + l / 2] = ((uint64_t)hi << 32) | r;
}

// Batched requests with 32 threads per stream: persistent warps take one chunk at a
// time from the counter (every level in one launch).  Lane 0 jumps the chunk to its
// start block with the single-thread table products; the warp then refills and emits as
// k_draw_warp does, one value per lane, with the multiplier of the chunk's level read
// from the level table.  For few, long chunks, where the latency of one refill is what
// counts.  TPB: threads per CTA (the block shape the tuner picks).
template <int TPB>
__global__ void __launch_bounds__(TPB)
    k_requests_warp(const BatchArgs b, const Item* __restrict__ items, uint64_t n_items, WorkCounters* wc) {
  __shared__ uint32_t scratch_s[TPB / 32][36];
  const unsigned l = lane_id();
  const int warp = threadIdx.x / 32;
  uint32_t* scratch = scratch_s[warp];
  while (true) {
    unsigned long long idx = 0;
    if (l == 0) idx = atomicAdd(&wc->next, 1ull);
    idx = __shfl_sync(kFull, idx, 0);
    if (idx >= n_items) break;
    const Item it = items[idx];
    if (l == 0) {  // the chunk's start state, on one thread
      uint32_t Ds[kLimbs], meta;
      request_state(b, it.req, Ds, meta);
      uint32_t c0 = meta_carry(meta);
      const uint32_t lv = meta_level(meta);
      if (it.jump) {  // X <- A^jump X
        uint32_t Xs[kLimbs];
        to_lcg(Ds, c0, Xs);
        bool have = true;
        apply_digits(b.s.table + (size_t)lv * kTableLimbs, 0, it.jump, Xs, have);
        to_ranlux(Xs, Ds);
        c0 = carry_of(Xs, Ds);
      }
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) scratch[k] = Ds[k];
      scratch[18] = c0;
      scratch[19] = lv;
    }
    __syncwarp();
    uint32_t D = l < 18 ? scratch[l] : 0u;
    uint32_t c = scratch[18];
    const uint32_t lvl = scratch[19];
    __syncwarp();  // scratch is free again (the conversion's rare case uses it)
    const uint32_t* luxl = b.s.lux + (size_t)lvl * kLimbs;
    auto A = [&](int k) { return __ldg(luxl + k); };
    const bool f64 = (it.info & 1u) != 0;
    const int need = f64 ? 2 : 1;
    const int per_block = kWords / need;
    const int64_t cnt = it.count, base = (int64_t)it.out;
    uint32_t pos = (it.info >> 8) & 0xFFu;
    // value of lane j of a block read from word w0 on (every lane takes part in the
    // shuffles; only lanes with a value store)
    auto emit = [&](int w0, int64_t idx0, int64_t nvals) {
      const int j = (int)l;
      if (f64) {
        const int w = w0 + 2 * j;
        const uint64_t v = wbits48(D, w < kWords - 1 ? w : 0);
        if (j < nvals && w + 2 <= kWords) b.out_f64[idx0 + j] = f64_bits_from48(v);
      } else {
        const int w = w0 + j;
        const uint32_t v = wword24(D, w < kWords ? w : 0);
        if (j < nvals && w < kWords) b.out_u24[idx0 + j] = v;
      }
    };
    int64_t k = 0;
    if (cnt > 0 && pos + need <= (uint32_t)kWords) {  // head of the start block
      const int64_t room = (kWords - pos) / need;
      const int64_t h = cnt < room ? cnt : room;
      emit((int)pos, base, h);
      k = h;
      pos += (uint32_t)(h * need);
    }
    if (k < cnt) {
      uint32_t X = wto_lcg(D, c);
#pragma unroll 1
      while (true) {
        uint32_t L, H;
        wmul(A, l < 18 ? X : 0u, L, H);
        X = wmod_m(L, H);
        D = wto_ranlux(X, scratch);
        const int64_t rem = cnt - k;
        if (rem >= per_block) {
          emit(0, base + k, per_block);
          k += per_block;
          pos = kWords;
          if (k == cnt) break;
        } else {
          emit(0, base + k, rem);
          k = cnt;
          pos = (uint32_t)(rem * need);
          break;
        }
      }
      c = wcarry(X, D);
    }
    if (b.advance && ((it.info >> 16) & 1u)) {  // last chunk of its request: final state
      const uint64_t st = b.req_stream[it.req];
      const uint32_t hiD = __shfl_down_sync(kFull, D, 1);
      if (l < 18 && (l & 1) == 0) b.s.D[(uint64_t)(l / 2) * b.s.stride + st] = ((uint64_t)hiD << 32) | D;
      if (l == 0) b.s.meta[st] = meta_pack(pos, c, lvl);
    }
  }
  finish_cta(wc);
}

template <int Kind>
cudaError_t launch_warp_kind(const DrawArgs& a, cudaStream_t st) {
  const unsigned grid = (unsigned)((a.s.n + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (a.uniform)
    k_draw_warp<Kind, true><<<grid, kWarpBlock, 0, st>>>(a);
  else
    k_draw_warp<Kind, false><<<grid, kWarpBlock, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_requests_warp(const BatchArgs& b, const Item* items, uint64_t n_items, WorkCounters* wc,
                                 unsigned grid, uint32_t tpb, cudaStream_t st) {
  if (n_items == 0) return cudaSuccess;
  if (tpb != 64 && tpb != 128 && tpb != 256) return cudaErrorInvalidValue;
  const uint64_t warps = tpb / 32;
  const uint64_t need = (n_items + warps - 1) / warps;
  if (grid > need) grid = (unsigned)need;
  if (tpb == 64) k_requests_warp<64><<<grid, 64, 0, st>>>(b, items, n_items, wc);
  else if (tpb == 256) k_requests_warp<256><<<grid, 256, 0, st>>>(b, items, n_items, wc);
  else k_requests_warp<128><<<grid, 128, 0, st>>>(b, items, n_items, wc);
  return cudaGetLastError();
}

cudaError_t launch_warp_test(int op, const uint64_t* in, uint64_t* out, uint32_t* carry, uint64_t n,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_test_warp<<<(unsigned)((n + kWarpsPerBlock - 1) / kWarpsPerBlock), kWarpBlock, 0, st>>>(op, in, out, carry, n);
  return cudaGetLastError();
}

bool warp_draw_supported(int kind) {
  return kind == kDrawU24 || kind == kDrawF64 || kind == kDrawF32 || kind == kDrawSumHist;
}

cudaError_t launch_draw_warp(int kind, const DrawArgs& a, cudaStream_t st) {
  if (a.s.n == 0) return cudaSuccess;
  switch (kind) {
    case kDrawU24: return launch_warp_kind<kDrawU24>(a, st);
    case kDrawF64: return launch_warp_kind<kDrawF64>(a, st);
    case kDrawSumHist: return launch_warp_kind<kDrawSumHist>(a, st);
    case kDrawF32: return launch_warp_kind<kDrawF32>(a, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace rlxpp
