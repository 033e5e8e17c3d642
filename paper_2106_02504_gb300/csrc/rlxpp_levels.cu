// Luxury-level setup, seeding, skipping, state import/export and the arithmetic test
// kernels.
//
// Seeding and skipping follow Sec. 2.4: exponentiation by squaring, here with a
// 4-bit fixed window whose powers A^(j 16^w) are tabulated once per luxury level, so
// that a stream needs one modular product per non-zero exponent digit.

#include "rlxpp_arith.cuh"
#include "rlxpp_fixmath.cuh"
#include "rlxpp_internal.h"
#include "rlxpp_state.cuh"

namespace rlxpp {
namespace {

// a = 2^-24 mod m = 2^576 - 2^552 - 2^240 + 2^216 + 1 (one recurrence step, Sec. 1),
// as 32-bit limbs, least significant first.
__constant__ uint32_t kOneStep[18] = {
    0x00000001u, 0x00000000u, 0x00000000u, 0x00000000u, 0x00000000u, 0x00000000u,
    0x01000000u, 0xFFFF0000u, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu,
    0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFEFFu};

// ---- per-level setup: A = a^p, then A^(16^w) by repeated squaring ----------------
__global__ void k_level_powers(uint32_t p, uint32_t* __restrict__ lux, uint32_t* __restrict__ table) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint32_t a[kLimbs], r[kLimbs], t[kLimbs];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) a[k] = kOneStep[k];
  // left-to-right square-and-multiply over the bits of p (p >= 1)
  int top = 31 - __clz(p);
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) r[k] = a[k];
#pragma unroll 1
  for (int b = top - 1; b >= 0; --b) {
    mul_mod(r, r, t);
    if ((p >> b) & 1u) {
      mul_mod(t, a, r);
    } else {
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) r[k] = t[k];
    }
  }
  store18(lux, r);
  // window w, digit 1: A^(16^w)
#pragma unroll 1
  for (int w = 0; w < kWindows; ++w) {
    store18(table + ((size_t)w * kDigits + 1) * kLimbs, r);
    if (w + 1 < kWindows) {
#pragma unroll 1
      for (int s = 0; s < 4; ++s) {
        mul_mod(r, r, t);
#pragma unroll
        for (int k = 0; k < kLimbs; ++k) r[k] = t[k];
      }
    }
  }
}

// digits 0 and 2..15 of every window: A^(j 16^w) = A^((j-1) 16^w) A^(16^w)
__global__ void k_level_digits(uint32_t* __restrict__ table) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= kWindows) return;
  uint32_t* row = table + (size_t)w * kDigits * kLimbs;
  uint32_t base[kLimbs], cur[kLimbs], t[kLimbs];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) {
    base[k] = row[kLimbs + k];
    cur[k] = base[k];
    row[k] = k == 0 ? 1u : 0u;
  }
#pragma unroll 1
  for (int j = 2; j < kDigits; ++j) {
    mul_mod(cur, base, t);
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) cur[k] = t[k];
    store18(row + (size_t)j * kLimbs, cur);
  }
}

// Seeding: stream i gets A^(2^96 seed_i), by the windowed table (at most 16 products
// for a 64-bit seed).  Each thread seeds kSeedRun consecutive streams; where a stream's
// seed is the previous stream's plus one at the same level, its state is the previous
// state times A^(2^96) (the table's window 24, digit 1): one product instead of one per
// nonzero hex digit of the seed.
constexpr int kSeedRun = 8;
__global__ void k_seed(StateView s, const uint64_t* __restrict__ seeds,
                       const uint8_t* __restrict__ level_of, uint32_t n_levels, bool keep_levels) {
  const uint64_t i0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) * kSeedRun;
  uint32_t X[kLimbs];
  uint64_t prev = 0;  // seed of the state in X, 0 when X holds none to continue from
  uint32_t prev_lvl = 0;
#pragma unroll 1
  for (int j = 0; j < kSeedRun; ++j) {
    const uint64_t i = i0 + j;
    if (i >= s.n) return;
    uint32_t lvl = keep_levels ? meta_level(s.meta[i]) : level_of ? level_of[i] : 0u;
    if (lvl >= n_levels) {
      set_status(s.status, RLXPP_ERR_INVALID);
      lvl = 0;
    }
    const uint64_t seed = seeds[i];
    const uint32_t* T = s.table + (size_t)lvl * kTableLimbs;
    if (seed == 0) {  // seeds start at 1: report, and leave a re-seeded stream as it was
      set_status(s.status, RLXPP_ERR_INVALID);
      prev = 0;
      if (keep_levels) continue;
      // a new handle's stream with seed 0: the state 1, so that it is defined
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) X[k] = k == 0 ? 1u : 0u;
    } else if (prev != 0 && seed == prev + 1 && lvl == prev_lvl) {
      uint32_t Y[kLimbs], R[kLimbs];
      load18(T + ((size_t)kSeedWindow0 * kDigits + 1) * kLimbs, Y);
      mul_mod(X, Y, R);
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) X[k] = R[k];
      prev = seed;
    } else {
      bool have = false;
      apply_digits(T, kSeedWindow0, seed, X, have);  // have: seed != 0
      prev = seed;
      prev_lvl = lvl;
    }
    uint32_t D[kLimbs];
    to_ranlux(X, D);
    store_state_D(s, i, D);
    s.meta[i] = meta_pack(0u, carry_of(X, D), lvl);
  }
}

__global__ void k_skip(StateView s, const uint64_t* __restrict__ n128) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const uint64_t lo = n128[2 * i], hi = n128[2 * i + 1];
  if ((lo | hi) == 0) return;
  const uint32_t meta = s.meta[i];
  const uint32_t lvl = meta_level(meta);
  const uint32_t* T = s.table + (size_t)lvl * kTableLimbs;
  uint32_t D[kLimbs], X[kLimbs];
  load_state_D(s, i, D);
  to_lcg(D, meta_carry(meta), X);
  bool have = true;  // X already holds the state: multiply by every digit's power
  apply_digits(T, 0, lo, X, have);
  apply_digits(T, 16, hi, X, have);
  to_ranlux(X, D);
  store_state_D(s, i, D);
  s.meta[i] = meta_pack(meta_pos(meta), carry_of(X, D), lvl);
}

// Position arithmetic of a draw of n values (need numbers each) without producing
// them: the rest of the current block, then whole blocks; X <- A^blocks X.
__global__ void k_skip_values(StateView s, const uint64_t* __restrict__ nvals, uint32_t need) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const uint64_t n = nvals[i];
  const uint32_t meta = s.meta[i];
  const uint32_t pos = meta_pos(meta), lvl = meta_level(meta);
  const uint64_t room = pos + need <= (uint32_t)kWords ? (kWords - pos) / need : 0;
  if (n <= room) {
    s.meta[i] = meta_pack(pos + (uint32_t)(n * need), meta_carry(meta), lvl);
    return;
  }
  const uint64_t rest = n - room, per = kWords / need;
  const uint64_t blocks = (rest - 1) / per + 1;
  const uint32_t new_pos = (uint32_t)((rest - (blocks - 1) * per) * need);
  uint32_t D[kLimbs], X[kLimbs];
  load_state_D(s, i, D);
  to_lcg(D, meta_carry(meta), X);
  bool have = true;
  apply_digits(s.table + (size_t)lvl * kTableLimbs, 0, blocks, X, have);
  to_ranlux(X, D);
  store_state_D(s, i, D);
  s.meta[i] = meta_pack(new_pos, carry_of(X, D), lvl);
}

__global__ void k_export(StateView s, const uint32_t* __restrict__ level_p, rlxpp_state* dst) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const uint32_t meta = s.meta[i];
  uint64_t* rec = reinterpret_cast<uint64_t*>(dst + i);
#pragma unroll
  for (int k = 0; k < 9; ++k) rec[k] = s.D[(uint64_t)k * s.stride + i];
  rec[9] = (uint64_t)meta_carry(meta) | ((uint64_t)meta_pos(meta) << 32);
  rec[10] = (uint64_t)level_p[meta_level(meta)];
}

__global__ void k_import(StateView s, const uint32_t* __restrict__ level_p, uint32_t n_levels,
                         const rlxpp_state* __restrict__ src) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const uint64_t* rec = reinterpret_cast<const uint64_t*>(src + i);
  uint32_t D[kLimbs];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint64_t v = rec[k];
    D[2 * k] = (uint32_t)v;
    D[2 * k + 1] = (uint32_t)(v >> 32);
  }
  const uint32_t carry = (uint32_t)rec[9], pos = (uint32_t)(rec[9] >> 32);
  const uint32_t p = (uint32_t)rec[10], reserved = (uint32_t)(rec[10] >> 32);
  uint32_t lvl = n_levels;
  for (uint32_t l = 0; l < n_levels; ++l)
    if (level_p[l] == p) { lvl = l; break; }
  bool ok = carry <= 1u && pos <= (uint32_t)kWords && reserved == 0u && lvl < n_levels;
  if (ok) {
    uint32_t X[kLimbs], D2[kLimbs];
    to_lcg(D, carry, X);
    uint32_t nz = 0;
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) nz |= X[k];
    // X < m  <=>  X + (2^240 - 1) < 2^576
    uint32_t e = add_cc(X[0], 0xFFFFFFFFu);
#pragma unroll
    for (int k = 1; k < 7; ++k) e = addc_cc(X[k], 0xFFFFFFFFu);
    e = addc_cc(X[7], 0xFFFFu);
#pragma unroll
    for (int k = 8; k < kLimbs; ++k) e = addc_cc(X[k], 0u);
    const uint32_t ge = addc(0u, 0u);
    (void)e;
    ok = nz != 0 && ge == 0;
    if (ok) {
      to_ranlux(X, D2);
      uint32_t diff = carry_of(X, D2) ^ carry;
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) diff |= D2[k] ^ D[k];
      ok = diff == 0;
    }
  }
  if (!ok) {
    set_status(s.status, RLXPP_ERR_INVALID);
    return;
  }
  store_state_D(s, i, D);
  s.meta[i] = meta_pack(pos, carry, lvl);
}

// ---- arithmetic unit tests --------------------------------------------------------
__device__ __forceinline__ void load_u64_limbs(const uint64_t* src, int n64, uint32_t* v) {
  for (int k = 0; k < n64; ++k) {
    v[2 * k] = (uint32_t)src[k];
    v[2 * k + 1] = (uint32_t)(src[k] >> 32);
  }
}
__device__ __forceinline__ void store_u64_limbs(uint64_t* dst, int n64, const uint32_t* v) {
  for (int k = 0; k < n64; ++k) dst[k] = ((uint64_t)v[2 * k + 1] << 32) | v[2 * k];
}

constexpr uint64_t kNaNBits = 0x7FF8000000000000ull;

__global__ void k_test(int op, const uint64_t* __restrict__ x, const uint64_t* __restrict__ y,
                       uint64_t* __restrict__ out, uint32_t* __restrict__ carry, uint64_t n) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t a[kLimbs], b[kLimbs], r[kLimbs], p[2 * kLimbs];
  switch (op) {
    case kTestMultiply:
      load_u64_limbs(x + 9 * i, 9, a);
      load_u64_limbs(y + 9 * i, 9, b);
      multiply9x9([&](int k) { return a[k]; }, b, p);
      store_u64_limbs(out + 18 * i, 18, p);
      break;
    case kTestModM:
      load_u64_limbs(x + 18 * i, 18, p);
      mod_m(p, r);
      store_u64_limbs(out + 9 * i, 9, r);
      break;
    case kTestMulMod:
      load_u64_limbs(x + 9 * i, 9, a);
      load_u64_limbs(y + 9 * i, 9, b);
      mul_mod(a, b, r);
      store_u64_limbs(out + 9 * i, 9, r);
      break;
    case kTestToRanlux:
      load_u64_limbs(x + 9 * i, 9, a);
      to_ranlux(a, r);
      store_u64_limbs(out + 9 * i, 9, r);
      carry[i] = carry_of(a, r);
      break;
    case kTestToLcg:
      load_u64_limbs(x + 9 * i, 9, a);
      to_lcg(a, carry[i], r);
      store_u64_limbs(out + 9 * i, 9, r);
      break;
    case kTestF64:
      out[i] = f64_bits_from48(x[i]);
      break;
    case kTestNegLn48: {  // w in [1, 2^48]; a NaN for anything else
      const uint64_t w = x[i];
      out[i] = (w >= 1 && w <= (1ull << 48))
                   ? (uint64_t)__double_as_longlong(fx_to_double(fx_neg_ln48(w), -120, false))
                   : kNaNBits;
      break;
    }
    case kTestCosSin2Pi48: {  // v < 2^48
      const bool ok = x[i] < (1ull << 48);
      const FxCosSin cs = fx_cos_sin_2pi48(ok ? x[i] : 0);
      out[2 * i] = ok ? (uint64_t)__double_as_longlong(fx_scale_to_double(1ull << 62, -62, cs.c, cs.nc)) : kNaNBits;
      out[2 * i + 1] = ok ? (uint64_t)__double_as_longlong(fx_scale_to_double(1ull << 62, -62, cs.s, cs.ns)) : kNaNBits;
      break;
    }
    case kTestBoxMuller48: {  // va, vb < 2^48
      double z0 = 0, z1 = 0;
      const bool ok = x[2 * i] < (1ull << 48) && x[2 * i + 1] < (1ull << 48);
      if (ok) fx_box_muller48(x[2 * i], x[2 * i + 1], z0, z1);
      out[2 * i] = ok ? (uint64_t)__double_as_longlong(z0) : kNaNBits;
      out[2 * i + 1] = ok ? (uint64_t)__double_as_longlong(z1) : kNaNBits;
      break;
    }
  }
}

inline unsigned grid_for(uint64_t n, unsigned block) {
  return (unsigned)((n + block - 1) / block);
}

}  // namespace

cudaError_t launch_level_setup(uint32_t p, uint32_t* lux_out18, uint32_t* table_out, cudaStream_t st) {
  k_level_powers<<<1, 32, 0, st>>>(p, lux_out18, table_out);
  k_level_digits<<<1, 64, 0, st>>>(table_out);
  return cudaGetLastError();
}

cudaError_t launch_seed(const StateView& s, const uint64_t* seeds, const uint8_t* level_of_stream,
                        uint32_t n_levels, bool keep_levels, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  k_seed<<<grid_for((s.n + kSeedRun - 1) / kSeedRun, 128), 128, 0, st>>>(s, seeds, level_of_stream, n_levels,
                                                                          keep_levels);
  return cudaGetLastError();
}

cudaError_t launch_skip(const StateView& s, const uint64_t* n128, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  k_skip<<<grid_for(s.n, 128), 128, 0, st>>>(s, n128);
  return cudaGetLastError();
}

cudaError_t launch_skip_values(const StateView& s, const uint64_t* n, uint32_t need, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  k_skip_values<<<grid_for(s.n, 128), 128, 0, st>>>(s, n, need);
  return cudaGetLastError();
}

cudaError_t launch_export(const StateView& s, const uint32_t* level_p, rlxpp_state* dst, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  k_export<<<grid_for(s.n, 256), 256, 0, st>>>(s, level_p, dst);
  return cudaGetLastError();
}

cudaError_t launch_import(const StateView& s, const uint32_t* level_p, uint32_t n_levels,
                          const rlxpp_state* src, cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  k_import<<<grid_for(s.n, 128), 128, 0, st>>>(s, level_p, n_levels, src);
  return cudaGetLastError();
}

cudaError_t launch_test(int which, const uint64_t* x, const uint64_t* y, uint64_t* out,
                        uint32_t* carry, uint64_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_test<<<grid_for(n, 128), 128, 0, st>>>(which, x, y, out, carry, n);
  return cudaGetLastError();
}

}  // namespace rlxpp

// ---- seeding without allocation ---------------------------------------------------
// A handle-free variant of k_seed for callers that must not allocate device memory.
// Its scratch (the multiplier and the power table of each requested luxury level) lives
// in one file-scope device array instead of memory from cudaMalloc.  The array exists
// on every GPU that loads the library, for the life of the process, and is shared by
// all calls: every call rewrites the tables it uses before reading them, and calls that
// overlap on the GPU (different streams, different threads) race on it.

namespace rlxpp {
namespace {

constexpr uint32_t kNoAllocMaxLevels = RLXPP_NOALLOC_MAX_LEVELS;
constexpr size_t kNoAllocLevelLimbs = 18 + kTableLimbs;  // A, then the power table

// 4 levels x (72 B + 46,080 B) = 184,608 bytes of device memory per GPU.
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocMaxLevels * kNoAllocLevelLimbs];

struct LevelList {
  uint32_t p[kNoAllocMaxLevels];
  uint32_t n;
};

// Seeds n streams straight into caller-owned state records (pos 0).  A stream whose
// level index is out of range gets an all-zero record (p = 0 marks it invalid).
__global__ void k_seed_records(const uint32_t* __restrict__ scratch, LevelList lv,
                               const uint64_t* __restrict__ seeds, const uint8_t* __restrict__ level_of,
                               uint64_t n, rlxpp_state* __restrict__ out) {
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t* rec = reinterpret_cast<uint64_t*>(out + i);
  const uint32_t lvl = level_of ? level_of[i] : 0u;
  const uint64_t seed = seeds[i];
  if (lvl >= lv.n || seed == 0) {  // invalid level index or seed: an all-zero record
#pragma unroll
    for (int k = 0; k < 11; ++k) rec[k] = 0;
    return;
  }
  const uint32_t* T = scratch + (size_t)lvl * kNoAllocLevelLimbs + 18;
  uint32_t X[kLimbs];
  bool have = false;
  apply_digits(T, kSeedWindow0, seed, X, have);
  uint32_t D[kLimbs];
  to_ranlux(X, D);
#pragma unroll
  for (int k = 0; k < 9; ++k) rec[k] = ((uint64_t)D[2 * k + 1] << 32) | D[2 * k];
  rec[9] = carry_of(X, D);          // pos 0
  rec[10] = lv.p[lvl];              // reserved 0
}

// Device address of g_noalloc_scratch in the current device's context, looked up on
// every call (a host-side query, no stream work), so that a context torn down and
// recreated between calls (cudaDeviceReset) never leaves a stale address behind.  The
// first lookup in a context may load the module, which a stream capture does not allow:
// hence the rule that the entry point runs once outside any capture first.
rlxpp_status noalloc_scratch(uint32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return set_last_error(RLXPP_ERR_CUDA, e != cudaSuccess ? cudaGetErrorString(e)
                                                          : "no device address for the scratch array");
  *out = static_cast<uint32_t*>(p);
  return RLXPP_OK;
}

// Memory the current device can dereference: its own device memory or managed memory.
// Device memory of another GPU is refused (without peer access a load from it faults).
bool device_pointer(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeManaged) return true;
  int cur = -1;
  if (attr.type != cudaMemoryTypeDevice || cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.device == cur;
}

}  // namespace
}  // namespace rlxpp

extern "C" rlxpp_status rlxpp_seed_states_noalloc(const uint32_t* levels, uint32_t n_levels,
                                                   const uint8_t* level_of_stream, const uint64_t* seeds,
                                                   uint64_t n_streams, rlxpp_state* out,
                                                   void* cuda_stream) {
  using namespace rlxpp;
  if (!levels || n_levels == 0)
    return set_last_error(RLXPP_ERR_INVALID, "need at least one luxury level");
  if (n_levels > kNoAllocMaxLevels)
    return set_last_error(RLXPP_ERR_INVALID,
                          "rlxpp_seed_states_noalloc: more luxury levels than its fixed scratch holds "
                          "(RLXPP_NOALLOC_MAX_LEVELS = 4)");
  LevelList lv{};
  lv.n = n_levels;
  for (uint32_t l = 0; l < n_levels; ++l) {
    if (levels[l] == 0) return set_last_error(RLXPP_ERR_INVALID, "luxury level must be >= 1");
    lv.p[l] = levels[l];
  }
  if (n_streams == 0) return RLXPP_OK;
  if (!seeds || !out) return set_last_error(RLXPP_ERR_INVALID, "null seeds or output");
  if (!device_pointer(seeds) || !device_pointer(out) ||
      (level_of_stream && !device_pointer(level_of_stream)))
    return set_last_error(RLXPP_ERR_INVALID,
                          "seeds, level indices and output must be memory of the current device");
  uint32_t* scratch = nullptr;
  if (rlxpp_status s = noalloc_scratch(&scratch)) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  for (uint32_t l = 0; l < n_levels; ++l) {
    uint32_t* base = scratch + (size_t)l * kNoAllocLevelLimbs;
    cudaError_t e = launch_level_setup(lv.p[l], base, base + 18, st);
    if (e != cudaSuccess) return set_last_error(RLXPP_ERR_CUDA, cudaGetErrorString(e));
  }
  k_seed_records<<<grid_for(n_streams, 128), 128, 0, st>>>(scratch, lv, seeds, level_of_stream, n_streams,
                                                           out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_last_error(RLXPP_ERR_CUDA, cudaGetErrorString(e));
  return RLXPP_OK;
}
