// The refill on the tensor cores (tcgen05, sm_103a): the product A X mod m of Sec. 2.1-2.2
// as an exact-integer fp16 matrix product.
//
// With X = sum_j x_j 2^(8j) (72 bytes) and R_j = A 2^(8j) mod m (72 bytes each),
//   A X = sum_j x_j R_j = sum_k S_k 2^(8k) (mod m),   S_k = sum_j x_j byte_k(R_j),
// so one refill of a tile of 128 streams is the product of a 128 x 72 byte matrix (the
// streams' X) with the 72 x 72 byte matrix of the level.  A stream's byte b enters as
// the fp16 subnormal b 2^-24 (its bit pattern is b itself, so writing the row is a byte
// shuffle), the level's bytes as fp16 integers; each product is b r 2^-24 with
// b r < 2^16, and every partial sum is a multiple of 2^-24 below
// (72 * 255^2 + 255) 2^-24 < 1/2, so fp32 accumulation is exact.  An extra K row
// (x_72 = 2048 against 2^-12) adds 1/2 to every column, so that the fp32 bit pattern of
// column k is the integer 0x3F000000 + S_k + e_k.  A second one (x_73 = 1 against
// e_k 2^-24, the bytes of a constant E) cancels those bias terms modulo m: the limb
// assembly below adds the bit patterns as they are, which leaves the bias
// C = 0x3F003F000000 sum_t 2^(32t) in the sum, and E = -C mod m.
// K = 80 and N = 80 after padding (five K = 16 instructions).
//
// One CTA owns one tile (128 threads, one stream per thread = one TMEM lane).  Per
// refill: each thread writes its X as fp16 into the shared A tile, one thread issues
// the five MMAs and commits them to an mbarrier, every thread waits (bounded) and loads
// its row of the fp32 accumulator from TMEM, forms the 590-bit sum of S_k 2^(8k), folds
// it below m (2^576 = 2^240 - 1 mod m) and continues with the conversion to RANLUX
// numbers (Sec. 2.3) and the output, as the integer-pipe kernels do.
//
// Shared operand layout (both operands K-major, no swizzle): core matrices of 8 rows x
// 16 bytes; element (row, k) of a 80-wide K tile sits at
//   (row / 8) * 1280 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2 bytes,
// i.e. leading-dimension byte offset (between K-adjacent core matrices) 128 and stride
// byte offset (between 8-row groups) 1280.
#include <cstring>

#include <cuda.h>  // CUtensorMap (the type only; the map is encoded on the host)
#include <cuda_fp16.h>

#include "rlxpp_arith.cuh"
#include "rlxpp_batch.h"
#include "rlxpp_drawloop.cuh"
#include "rlxpp_internal.h"
#include "rlxpp_state.cuh"

namespace rlxpp {
namespace {

constexpr int kTcRows = 128;                 // streams per tile = TMEM lanes = M
constexpr int kTcK = 80;                     // 72 bytes + bias + padding
constexpr int kTcN = 80;                     // 72 output columns + padding
constexpr int kTileBytes = kTcRows * kTcK * 2;   // 20480
constexpr int kBBytes = kTcN * kTcK * 2;         // 12800
constexpr int kLBO = 128, kSBO = 1280;
constexpr uint64_t kWaitLimit = 1ull << 22;  // mbarrier polls (about 0.3 s) before giving up

// fp16 element offset of (row, k) in a K-major 80-wide tile
__host__ __device__ constexpr int tc_off(int row, int k) {
  return (row >> 3) * (kSBO / 2) + (k >> 3) * (kLBO / 2) + (row & 7) * 8 + (k & 7);
}

// ---- PTX wrappers ----------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;  // the common case, outside the loop
  for (uint32_t i = 0; i < (uint32_t)kWaitLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// whole warp: allocate ncols TMEM columns, address written to *dst (shared)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  // start address, LBO and SBO in 16-byte units; version 1 (bits 46-47); no swizzle
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         (1ull << 46);
}
// kind::f16 instruction descriptor: D f32, A and B f16, both K-major, N = 80, M = 128
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}
// whole warp: 64 consecutive columns of this warp's 32 lanes into registers
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// The product with the A operand in tensor memory (a_tmem: its first column, lane 0).
__device__ __forceinline__ void tc_mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}
// whole warp: 32 (4) consecutive columns of this warp's 32 lanes from registers
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
      "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
      "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
      "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ---- per-thread pieces -------------------------------------------------------------
// X (18 limbs) -> 72 fp16 values (one per byte) in this thread's row of the A tile
// (chunks 0..8 of the row, 16 bytes each).  The half with bit pattern b (< 2^10) is the
// subnormal b 2^-24, exact: each pair of bytes is one byte shuffle with zeros.
__device__ __forceinline__ void write_x_row(__half* tile, int row, const uint32_t X[kLimbs]) {
  uint4* base = reinterpret_cast<uint4*>(tile + tc_off(row, 0));
#pragma unroll
  for (int c = 0; c < 9; ++c) {  // chunk c = bytes 8c .. 8c+7 = limbs 2c, 2c+1
    const uint32_t L0 = X[2 * c], L1 = X[2 * c + 1];
    base[c * (kLBO / 16)] = make_uint4(__byte_perm(L0, 0u, 0x4140u), __byte_perm(L0, 0u, 0x4342u),
                                       __byte_perm(L1, 0u, 0x4140u), __byte_perm(L1, 0u, 0x4342u));
  }
}

// Column bit patterns 0x3F000000 + S_k + e_k -> the assembled value X + T 2^576, which
// is congruent to sum_k S_k 2^(8k) mod m.
__device__ __forceinline__ void columns_assemble(const uint32_t col[72], uint32_t X[kLimbs], uint32_t& T) {
  // Limb t gathers its four columns as w_t = u + 2^16 v (below 2^48, as lo + hi 2^32),
  // u = col_4t + 2^8 col_4t+1 mod 2^32 = 0x3F000000 + (S + e)_4t + 2^8 (S + e)_4t+1
  // exactly (2^8 0x3F000000 = 0 mod 2^32 and the rest stays below 2^32), v likewise:
  // w_t = 0x3F003F000000 + sum_i (S + e)_4t+i 2^(8i), whose bias part E cancels mod m.
  uint32_t lo[kLimbs], hi[kLimbs];
#pragma unroll
  for (int t = 0; t < kLimbs; ++t) {
    uint32_t u, v;  // multiply-adds on the FMA pipe
    asm("mad.lo.u32 %0, %1, 256, %2;" : "=r"(u) : "r"(col[4 * t + 1]), "r"(col[4 * t]));
    asm("mad.lo.u32 %0, %1, 256, %2;" : "=r"(v) : "r"(col[4 * t + 3]), "r"(col[4 * t + 2]));
    const uint64_t w = mad_wide(v, 65536u, (uint64_t)u);
    lo[t] = lo32(w);
    hi[t] = hi32(w);
  }
  // value = sum_t lo_t 2^(32t) + hi_t 2^(32(t+1)): one carry chain, top limb T; the
  // value is S + E + C with S < 2^590.2, E < 2^576 and C = 0x3F003F sum_t 2^(32t + 8),
  // so 16128 <= T <= 34489
  X[0] = lo[0];
  X[1] = add_cc(lo[1], hi[0]);
#pragma unroll
  for (int t = 2; t < kLimbs; ++t) X[t] = addc_cc(lo[t], hi[t - 1]);
  T = addc(hi[kLimbs - 1], 0u);
}

// The fold of the assembled value, X + T (2^240 - 1) with 16128 <= T <= 34489, and the
// final correction into [0, m).
__device__ __forceinline__ void fold_x(uint32_t X[kLimbs], uint32_t T) {
  // fold: X + T (2^240 - 1).  T (2^240 - 1) = (T - 1) 2^240 + (2^240 - T) for 1 <= T < 2^16:
  // limb 0 = 2^32 - T, limbs 1..6 all ones, limb 7 = ((T - 1) << 16) | 0xFFFF.
  X[0] = add_cc(X[0], 0u - T);
#pragma unroll
  for (int k = 1; k < 7; ++k) X[k] = addc_cc(X[k], 0xFFFFFFFFu);
  X[7] = addc_cc(X[7], (T - 1u) << 16 | 0xFFFFu);
  X[8] = addc_cc(X[8], 0u);
  // a carry out of limb 8 needs that limb all ones before (rare): only then run the
  // rest of the chain, and past limb 17 it is another 2^576 while the low part is
  // below 2^256, so 2^240 - 1 is added again
  if (__builtin_expect(addc(0u, 0u) != 0u, 0)) {
    X[9] = add_cc(X[9], 1u);
#pragma unroll
    for (int k = 10; k < kLimbs; ++k) X[k] = addc_cc(X[k], 0u);
    if (addc(0u, 0u)) {
      X[0] = add_cc(X[0], 0xFFFFFFFFu);
#pragma unroll
      for (int k = 1; k < 7; ++k) X[k] = addc_cc(X[k], 0xFFFFFFFFu);
      X[7] = addc(X[7], 0xFFFFu);
    }
  }
  // X >= m needs bits 240..575 all set (rare, so the top limb is tested first): then
  // X - m = X + 2^240 - 1 mod 2^576
  if (__builtin_expect(X[17] == 0xFFFFFFFFu, 0)) {
    const uint32_t top = X[8] & X[9] & X[10] & X[11] & X[12] & X[13] & X[14] & X[15] & X[16];
    if (top == 0xFFFFFFFFu && X[7] >= 0xFFFF0000u) {
      uint32_t e[kLimbs];
      e[0] = add_cc(X[0], 0xFFFFFFFFu);
#pragma unroll
      for (int k = 1; k < 7; ++k) e[k] = addc_cc(X[k], 0xFFFFFFFFu);
      e[7] = addc_cc(X[7], 0xFFFFu);
#pragma unroll
      for (int k = 8; k < kLimbs; ++k) e[k] = addc_cc(X[k], 0u);
      const uint32_t ge = addc(0u, 0u);
#pragma unroll
      for (int k = 0; k < kLimbs; ++k) X[k] = ge ? e[k] : X[k];
    }
  }
}

// Column bit patterns 0x3F000000 + S_k + e_k -> X = sum_k S_k 2^(8k) mod m.
__device__ __forceinline__ void columns_to_x(const uint32_t col[72], uint32_t X[kLimbs]) {
  uint32_t T;
  columns_assemble(col, X, T);
  fold_x(X, T);
}

// The integer epilogue of one refill: X = sum_k S_k 2^(8k) mod m from the column bit
// patterns, written to this thread's operand row (the next product's input), and
// D = its 24 RANLUX numbers (Sec. 2.3).  The common case is computed without a branch:
// the fold's limb 0 does not borrow and its carry stops in limb 8, the top limb is not
// all ones (so X < m) and the conversion's quick test (that of to_ranlux) decides its
// quotient, with no carry out of limb 7 of X + q.
// Any other case (about 2^-15 of the refills) is redone in one branch by the exact forms
// (fold_x, to_ranlux), which rewrite the row and D.
__device__ __forceinline__ void tc_epilogue(const uint32_t col[72], __half* tile, int row, uint32_t X[kLimbs],
                                            uint32_t D[kLimbs]) {
  uint32_t Xa[kLimbs], T;
  columns_assemble(col, Xa, T);
  // the fold X + T (2^240 - 1) = X + (T - 1) 2^240 + (2^32 - T) + sum_(0<k<7) 0xFFFFFFFF 2^(32k)
  // + 0xFFFF 2^224 when limb 0 does not borrow (Xa_0 >= T, about all but 2^-17 of the
  // refills): limbs 1..6 then come out unchanged and limb 7 gains T 2^16, so the chain
  // is two limbs long
  const bool b0 = Xa[0] < T;
  X[0] = Xa[0] - T;
#pragma unroll
  for (int k = 1; k < 7; ++k) X[k] = Xa[k];
  X[7] = add_cc(Xa[7], T << 16);
  X[8] = addc_cc(Xa[8], 0u);
  const uint32_t c9 = addc(0u, 0u);  // carry out of limb 8
#pragma unroll
  for (int k = 9; k < kLimbs; ++k) X[k] = Xa[k];
  write_x_row(tile, row, X);
  const uint32_t t15 = sub_cc(__funnelshift_l(X[7], X[8], 16), X[15]);
  const uint32_t t16 = subc_cc(__funnelshift_l(X[8], X[9], 16), X[16]);
  const uint32_t t17 = subc_cc(__funnelshift_l(X[9], X[10], 16), X[17]);
  const uint32_t borrow = subc(0u, 0u) & 1u;
  const uint32_t q0 = __funnelshift_l(X[10], X[11], 16);
  D[0] = add_cc(X[0], q0 - borrow);
#pragma unroll
  for (int k = 1; k < 7; ++k) D[k] = addc_cc(X[k], __funnelshift_l(X[10 + k], X[11 + k], 16));
  D[7] = addc_cc(X[7], X[17] >> 16);
  const uint32_t c8 = addc(0u, 0u);  // carry out of limb 7 of X + q
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) D[k] = X[k];
  const bool rare = b0 || (c9 | c8) != 0u || X[17] == 0xFFFFFFFFu || (t15 & t16 & t17) == 0xFFFFFFFFu ||
                    (t15 | t16 | t17) == 0u || q0 < borrow;
  if (__builtin_expect(rare, 0)) {
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) X[k] = Xa[k];
    fold_x(X, T);
    write_x_row(tile, row, X);
    to_ranlux(X, D);
  }
}

struct TcShared {
  uint64_t bar;      // MMA completion
  uint32_t taddr;    // TMEM base (group 0's copy is the CTA's)
  uint32_t pos0;     // read position of the tile's first stream at entry
};
constexpr int kSharedBytes = 128;              // TcShared, padded (keeps the staging 128-byte aligned)
constexpr int kStageBytes = 96;                // one block of output per thread

// Shared memory of a CTA of T tile-groups (128 threads and one tile each): the level's
// matrix once, then per group its A tile, its TcShared and, for kernels that write
// values, its [128][96 B] output staging box.  Groups start on 1 KB boundaries.
constexpr int kBRegion = 13 * 1024;                          // kBBytes rounded up
constexpr int kGroupStage = kTileBytes + kSharedBytes;       // 20608, a multiple of 128
constexpr int kGroupBytesOut = 33 * 1024;                    // >= kGroupStage + 128 * 96
constexpr int kGroupBytesNoOut = 21 * 1024;                  // >= kGroupStage
static_assert(kBRegion >= kBBytes && kGroupBytesOut >= kGroupStage + kTcRows * kStageBytes &&
                  kGroupBytesNoOut >= kGroupStage && kGroupStage % 128 == 0,
              "shared memory layout");
__host__ __device__ constexpr int tc_smem_bytes(int groups, bool staging) {
  return kBRegion + groups * (staging ? kGroupBytesOut : kGroupBytesNoOut);
}
// TMEM: one allocation per CTA; group g's 80 accumulator columns start at column 96 g
// (a multiple of the 32-column allocation unit), so five groups fit in 512 columns.
constexpr int kGroupCols = 96;
__host__ __device__ constexpr uint32_t tc_alloc_cols(int groups) { return groups == 1 ? 128u : 512u; }
static_assert(4 * kGroupCols + kTcN <= 512, "five groups' accumulators in 512 TMEM columns");

// This thread's tile-group: group index g (barrier g + 1), row t of the group's tile.
// The group's lead thread (lane 0 of its warp g mod 4) issues its MMAs, so that the
// groups' issuing warps sit on different SM sub-partitions; tile-wide stores are issued
// by row 0, which is live whenever any row of the tile is.
struct TcGroup {
  int g, t, lead;
  __half* tile;
  TcShared* sh;
  unsigned char* stage;  // the group's staging box (kernels that write values)
};
__device__ __forceinline__ TcGroup tc_group(unsigned char* smem, bool staging) {
  TcGroup G;
  G.g = threadIdx.x / kTcRows;
  G.t = threadIdx.x % kTcRows;
  G.lead = (G.g % 4) * 32;
  unsigned char* base = smem + kBRegion + G.g * (staging ? kGroupBytesOut : kGroupBytesNoOut);
  G.tile = reinterpret_cast<__half*>(base);
  G.sh = reinterpret_cast<TcShared*>(base + kTileBytes);
  G.stage = base + kGroupStage;
  return G;
}
__device__ __forceinline__ __half* tc_bmat(unsigned char* smem) { return reinterpret_cast<__half*>(smem); }

// Barriers of one group (128 threads, warp-uniform): named barrier g + 1.
__device__ __forceinline__ void group_sync(const TcGroup& G) {
  asm volatile("bar.sync %0, 128;" ::"r"(G.g + 1) : "memory");
}
__device__ __forceinline__ bool group_or(const TcGroup& G, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.or.pred b, %2, 128, a;\n selp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(G.g + 1)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ bool group_and(const TcGroup& G, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n bar.red.and.pred b, %2, 128, a;\n selp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(G.g + 1)
      : "memory");
  return r != 0;
}

// A full block of output (12 doubles or 24 numbers, 96 bytes) from this thread's
// staging slot to global memory by one bulk copy (the TMA engine writes it), after the
// slot's previous copy has been read out.  gdst must be 16-byte aligned.
__device__ __forceinline__ void bulk_store96(void* gdst, uint4* slot, const uint4 v[6]) {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 6; ++q) slot[q] = v[q];
  fence_proxy_async_smem();
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], 96;" ::"l"(gdst), "r"(smem_addr(slot))
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// A tile-wide store of one block per stream: the staging area holds the 128 threads'
// 96-byte blocks as a dense [128][96 B] box, which one TMA tensor store writes to rows
// y .. y + 127 at column x of the output (rows past the stream count and columns past
// the count per stream are clipped by the tensor map's extents).  One thread issues
// it after the CTA barrier that follows the writes, and waits for the copy to have
// read the staging area before the barrier that precedes the next writes.
struct TileStore {
  const CUtensorMap* map = nullptr;  // null: no tile-wide stores in this launch
  uint32_t src = 0;                  // shared address of the staging box
  int x = 0, y = 0;
  bool pending = false;              // a written box waits to be stored (thread 0's view)
};
__device__ __forceinline__ void tile_store_issue(TileStore& t) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(t.map)),
               "r"(t.x), "r"(t.y), "r"(t.src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  t.pending = false;
}

template <int Kind>
__device__ __forceinline__ void block_values(const uint32_t D[kLimbs], uint4 v[6]) {
  if constexpr (Kind == kDrawF64) {
    block_f64(D, v);
  } else if constexpr (Kind == kDrawF32) {
#pragma unroll
    for (int q = 0; q < 6; ++q)
      v[q] = make_uint4(f32_bits_from24(word24(D, 4 * q)), f32_bits_from24(word24(D, 4 * q + 1)),
                        f32_bits_from24(word24(D, 4 * q + 2)), f32_bits_from24(word24(D, 4 * q + 3)));
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q)
      v[q] = make_uint4(word24(D, 4 * q), word24(D, 4 * q + 1), word24(D, 4 * q + 2), word24(D, 4 * q + 3));
  }
}

// Group 0's TcShared: its taddr is the CTA's TMEM base.
__device__ __forceinline__ TcShared* tc_sh0(unsigned char* smem) {
  return reinterpret_cast<TcShared*>(smem + kBRegion + kTileBytes);
}

// Setup of a CTA of `groups` tile-groups: the level's matrix into shared memory (unless
// bimg is null: the kernel loads it later), the constant chunk 9 of every tile row
// (2048 and 1 at k = 72, 73, zeros after), one mbarrier per group and the CTA's TMEM
// columns.  Ends with a CTA barrier.
__device__ __forceinline__ void tc_setup(unsigned char* smem, const TcGroup& G, const __half* __restrict__ bimg,
                                         int groups) {
  const int tid = threadIdx.x;
  if (bimg) {
    const uint4* src = reinterpret_cast<const uint4*>(bimg);
    uint4* dst = reinterpret_cast<uint4*>(tc_bmat(smem));
    for (int i = tid; i < kBBytes / 16; i += groups * kTcRows) dst[i] = src[i];
  }
  {
    __half* row9 = G.tile + tc_off(G.t, 72);
    row9[0] = __float2half(2048.f);
    row9[1] = __float2half(1.f);
#pragma unroll
    for (int k = 2; k < 8; ++k) row9[k] = __float2half(0.f);
  }
  if (G.t == G.lead) {
    mbar_init(&G.sh->bar, 1);
    fence_barrier_init();
  }
  if (tid < 32) tmem_alloc(&tc_sh0(smem)->taddr, tc_alloc_cols(groups));
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// TMEM address of the group's accumulator (lane 0, its first column).
__device__ __forceinline__ uint32_t tc_tmem(unsigned char* smem, const TcGroup& G) {
  return tc_sh0(smem)->taddr + (uint32_t)(G.g * kGroupCols);
}

// Publish this thread's row to the tensor core: the fences and the group's barrier
// before the MMA; returns whether any thread of the group's tile still refills.
__device__ __forceinline__ bool tc_publish(const TcGroup& G, bool mine) {
  fence_proxy_async_smem();  // this thread's row writes -> visible to the tensor core
  tc_fence_before();
  const bool any = group_or(G, mine);
  tc_fence_after();
  return any;
}

// One refill of the group's tile, its rows published (tc_publish); returns false on a
// wait timeout.  issue = false leaves the barrier without an arrival (used to test the
// timeout path).  With a store, the group's first thread also issues the pending
// tile-wide store behind the MMA and waits for it to have read the staging box.
__device__ __forceinline__ bool tc_refill_after_publish(const TcGroup& G, const __half* bmat, uint32_t taddr,
                                                        uint32_t& phase, uint32_t col[72], bool issue = true,
                                                        TileStore* store = nullptr) {
  if (G.t == G.lead && issue) {
    const uint32_t a0 = smem_addr(G.tile), b0 = smem_addr(bmat);
#pragma unroll
    for (int s = 0; s < kTcK / 16; ++s)  // K = 16 per instruction: two core matrices
      tc_mma(taddr, smem_desc(a0 + s * 2 * kLBO), smem_desc(b0 + s * 2 * kLBO), s > 0 ? 1u : 0u);
    tc_commit(&G.sh->bar);
  }
  // the previous refill's blocks, written before the publishing barrier
  if (store && G.t == 0 && store->pending) tile_store_issue(*store);
  const bool ok = mbar_wait_bounded(&G.sh->bar, phase);
  if (store && G.t == 0) bulk_wait_read_all();  // staging free again after the next barrier
  if (!group_and(G, ok)) return false;           // phase stays: the teardown waits on it
  phase ^= 1u;
  tc_fence_after();
  // warp (t / 32) of the group reads TMEM lanes 32 (t / 32) .. + 31, its rows
  const uint32_t lane_addr = taddr + ((uint32_t)((G.t / 32) * 32) << 16);
#pragma unroll
  for (int q = 0; q < 4; ++q) tmem_ld16(lane_addr + 16 * q, col + 16 * q);
  tmem_ld8(lane_addr + 64, col + 64);
  tmem_wait_ld();
  return true;
}

__device__ __forceinline__ bool tc_refill(const TcGroup& G, const __half* bmat, uint32_t taddr, uint32_t& phase,
                                          uint32_t col[72], bool issue = true) {
  tc_publish(G, true);
  return tc_refill_after_publish(G, bmat, taddr, phase, col, issue);
}

// Release the CTA's TMEM columns.  After a timed-out wait (pending), first wait once
// more, again with a limit, for the MMA that may still be writing them.  Every thread
// of the CTA calls it.
__device__ __forceinline__ void tc_teardown(unsigned char* smem, const TcGroup& G, bool pending, uint32_t phase,
                                            int groups) {
  if (pending) (void)mbar_wait_bounded(&G.sh->bar, phase);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(tc_sh0(smem)->taddr, tc_alloc_cols(groups));
}

// The full blocks of one warp (96 bytes per lane that has one; dst = 0 marks a lane
// without) written cooperatively: each lane's block is already in its staging slot (the
// warp's 32 slots are contiguous), and store i of lane l writes unit i 32 + l of the
// warp's 3072 staged bytes to its block's destination, so one store instruction covers
// 256 (or 128) consecutive bytes of one to three blocks instead of 32 scattered pieces.
// 8-byte units when every destination is 8-byte aligned, else 4-byte units.  Every lane
// of the warp calls it.
__device__ __forceinline__ void warp_store_blocks(const unsigned char* wstage, uint64_t dst) {
  const unsigned lane = threadIdx.x & 31u;
  __syncwarp();  // the lanes' slots are written
  if (__all_sync(0xFFFFFFFFu, (dst & 7u) == 0)) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(wstage);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const unsigned u = i * 32u + lane;  // = 12 t + w: unit w of lane t's block
      const unsigned t = u / 12u, w = u - 12u * t;
      const uint64_t p = __shfl_sync(0xFFFFFFFFu, dst, (int)t);
      const uint64_t val = src[u];
      if (p) reinterpret_cast<uint64_t*>(p)[w] = val;
    }
  } else {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wstage);
#pragma unroll 4
    for (int i = 0; i < 24; ++i) {
      const unsigned u = i * 32u + lane;  // = 24 t + w
      const unsigned t = u / 24u, w = u - 24u * t;
      const uint64_t p = __shfl_sync(0xFFFFFFFFu, dst, (int)t);
      const uint32_t val = src[u];
      if (p) reinterpret_cast<uint32_t*>(p)[w] = val;
    }
  }
  __syncwarp();  // the slots may be written again
}

// The full blocks of one warp of strided chunks (one request's blocks f .. f + 31 of a
// refill): lanes 0 .. n - 1 have full blocks whose destinations run on consecutively
// (lane l's is lane 0's plus 96 l bytes) and the others none, so the warp copies its
// n * 96 staged bytes as one contiguous run, 16-, 8- or 4-byte units by the alignment of
// its start.  Destinations that do not form such a run (not expected) go through
// warp_store_blocks.  Every lane of the warp calls it.
__device__ __forceinline__ void warp_store_run(const unsigned char* wstage, uint64_t dst) {
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t d0 = __shfl_sync(0xFFFFFFFFu, dst, 0);
  const unsigned nfull = __popc(__ballot_sync(0xFFFFFFFFu, dst != 0));
  const bool in_run = dst == 0 ? lane >= nfull : (lane < nfull && dst == d0 + (uint64_t)kStageBytes * lane);
  if (!__all_sync(0xFFFFFFFFu, in_run)) {
    warp_store_blocks(wstage, dst);
    return;
  }
  __syncwarp();  // the lanes' slots are written
  if ((d0 & 15u) == 0) {
    const uint4* src = reinterpret_cast<const uint4*>(wstage);
    uint4* o = reinterpret_cast<uint4*>(d0);
    const unsigned n = nfull * (kStageBytes / 16);
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (i * 32u + lane < n) o[i * 32u + lane] = src[i * 32u + lane];
  } else if ((d0 & 7u) == 0) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(wstage);
    uint64_t* o = reinterpret_cast<uint64_t*>(d0);
    const unsigned n = nfull * (kStageBytes / 8);
#pragma unroll
    for (int i = 0; i < 12; ++i)
      if (i * 32u + lane < n) o[i * 32u + lane] = src[i * 32u + lane];
  } else {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(wstage);
    uint32_t* o = reinterpret_cast<uint32_t*>(d0);
    const unsigned n = nfull * (kStageBytes / 4);
#pragma unroll
    for (int i = 0; i < 24; ++i)
      if (i * 32u + lane < n) o[i * 32u + lane] = src[i * 32u + lane];
  }
  __syncwarp();  // the slots may be written again
}

// Draw kernel on the tensor path (single-level handles).  Same semantics as k_draw.
// A CTA holds T tile-groups (one SM's worth), each refilling its own tile of 128
// streams independently of the others.  tmap (when use_tma): the output as a
// [n][count_each] tensor of 4- or 8-byte elements with a [128][per block] box, for the
// tile-wide stores of tiles whose streams move in step.
// Coop: the launch has no tensor map (use_tma = 0) and every tile writes its blocks by
// warp-cooperative stores; otherwise tiles out of step copy each lane's block by a bulk
// copy (this form keeps the registers of the tile-store path free).
template <int Kind, int T, bool Coop>
__global__ void __launch_bounds__(kTcRows* T, T == 1 ? 4 : 1)
    k_draw_tc(const DrawArgs a, const __half* __restrict__ bimg, const __grid_constant__ CUtensorMap tmap,
              int use_tma) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr bool kStaging = Kind != kDrawSumHist;
  const TcGroup G = tc_group(smem, kStaging);
  const __half* bmat = tc_bmat(smem);
  uint4* slot = reinterpret_cast<uint4*>(G.stage + G.t * kStageBytes);
  const unsigned char* wstage = G.stage + (G.t & ~31) * kStageBytes;  // this warp's 32 slots
  __shared__ unsigned int hist_s[Kind == kDrawSumHist ? 4 * T * 256 : 1];  // one histogram per warp
  const int tid = threadIdx.x;
  if (Kind == kDrawSumHist)
    for (int t = tid; t < 4 * T * 256; t += kTcRows * T) hist_s[t] = 0;
  tc_setup(smem, G, bimg, T);
  const uint32_t taddr = tc_tmem(smem, G);

  const StateView& s = a.s;
  const uint64_t tile_idx = (uint64_t)blockIdx.x * T + G.g;
  const uint64_t i = tile_idx * kTcRows + G.t;
  const bool live = i < s.n;
  int64_t cnt = 0, base = 0;
  uint32_t pos = kWords, c = 0, lvl = 0;
  uint32_t D[kLimbs];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) D[k] = 0;
  if (live) {
    if (a.counts) {
      cnt = a.counts[i];
      base = a.offsets[i];
    } else {
      cnt = a.count_each;
      base = (int64_t)i * a.count_each;
    }
    const uint32_t meta = s.meta[i];
    pos = meta_pos(meta);
    c = meta_carry(meta);
    lvl = meta_level(meta);
    load_state_D(s, i, D);
  }
  Consumer<Kind> out;
  if constexpr (Kind == kDrawU24) out.out = static_cast<uint32_t*>(a.out);
  if constexpr (Kind == kDrawF64) out.out = static_cast<uint64_t*>(a.out);
  if constexpr (Kind == kDrawF32) out.out = static_cast<uint32_t*>(a.out);
  if constexpr (Kind == kDrawSumHist) {
    out.sum = 0;
    out.hist = hist_s + (tid / 32) * 256;
  }
  if constexpr (Kind == kDrawExp) out.out = static_cast<double*>(a.out);
  if constexpr (Kind == kDrawNormal) {  // n normals take 2 ceil(n / 2) doubles
    out.out = static_cast<double*>(a.out);
    out.base = base;
    out.end = base + cnt;
    out.va = 0;
    cnt += cnt & 1;
  }
  constexpr int need = (Kind == kDrawU24 || Kind == kDrawF32) ? 1 : 2;
  constexpr int per_block = kWords / need;
  const uint32_t pos_in = pos;
  int64_t k = 0;
  if (live && cnt > 0 && pos + need <= (uint32_t)kWords) {  // head of the current block
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
  bool mine = live && k < cnt;
  uint32_t X[kLimbs];
  to_lcg(D, c, X);
  // Tile-wide stores when every live stream of the tile starts at the tile's first
  // position (then, with one count for all, they stay in step) and the first column
  // after the head is 16-byte aligned.  The group's thread 0 decides for the tile (it
  // is live whenever any thread of the group is).
  TileStore store;
  bool tma = false;
  if constexpr (Kind != kDrawSumHist && !Coop) {
    if (use_tma) {  // uniform over the grid
      if (G.t == 0) G.sh->pos0 = pos_in;
      group_sync(G);
      const bool same = !live || (pos_in == G.sh->pos0 && ((k * (int64_t)(need * 4)) & 15) == 0);
      tma = group_and(G, same);
      store.map = &tmap;
      store.src = smem_addr(G.stage);
      store.y = (int)(tile_idx * kTcRows);
    }
  }
  uint32_t phase = 0;
  bool ok = true;
  bool stored = false;  // this stream's final state is written
  // A stream's state lives in its operand row between refills: each new X is written
  // there as soon as it is formed (the product that read the tile is complete), and the
  // final (D, carry) is stored when the stream's last block is drawn, so neither X nor
  // D stays live across the wait for the next product.
  write_x_row(G.tile, G.t, X);
  while (true) {
    if (!tc_publish(G, mine)) break;  // every stream of the tile is done
    uint32_t col[72];
    if (!tc_refill_after_publish(G, bmat, taddr, phase, col, true, tma ? &store : nullptr)) {
      ok = false;
      break;
    }
    uint64_t dst = 0;  // destination of this lane's full block (streams out of step)
    if (mine) {
      tc_epilogue(col, G.tile, G.t, X, D);  // X also into the next product's operand row
      const int64_t rem = cnt - k;
      if (tma) {
        // the whole block into this thread's row of the staging box; past the count
        // the box is clipped
        uint4 v[6];
        block_values<Kind>(D, v);
#pragma unroll
        for (int q = 0; q < 6; ++q) slot[q] = v[q];
        fence_proxy_async_smem();
        store.x = (int)k;
        store.pending = true;
        if (rem >= per_block) {
          k += per_block;
          pos = kWords;
        } else {
          k = cnt;
          pos = (uint32_t)(rem * need);
        }
      } else if (rem >= per_block) {
        if constexpr (Kind == kDrawSumHist || Kind == kDrawNormal || Kind == kDrawExp) {
          out.block(D, base + k);
        } else if constexpr (Coop) {
          // staged here, written by the whole warp below
          uint4 v[6];
          block_values<Kind>(D, v);
#pragma unroll
          for (int q = 0; q < 6; ++q) slot[q] = v[q];
          dst = reinterpret_cast<uint64_t>(out.out + base + k);
        } else {
          // streams out of step in a launch with tile-wide stores: a bulk copy of this
          // lane's block from its staging slot
          void* gdst = out.out + base + k;
          if ((reinterpret_cast<uintptr_t>(gdst) & 15) == 0) {
            uint4 v[6];
            block_values<Kind>(D, v);
            bulk_store96(gdst, slot, v);
          } else {
            out.block(D, base + k);
          }
        }
        k += per_block;
        pos = kWords;
      } else {
        out.partial(D, base + k, rem);
        k = cnt;
        pos = (uint32_t)(rem * need);
      }
      mine = k < cnt;
      if (!mine) {
        c = carry_of(X, D);
        store_state_D(s, i, D);
        stored = true;
      }
    }
    if constexpr (Coop) warp_store_blocks(wstage, dst);
  }
  if (tma && G.t == 0 && store.pending) tile_store_issue(store);  // the last blocks
  if (Kind != kDrawSumHist) bulk_wait_all();  // this thread's output copies are done
  // after a timed-out wait, streams that finished keep their new state (D with its
  // position and carry), the others their old one
  if (live && (ok || stored)) s.meta[i] = meta_pack(pos, c, lvl);
  if (!ok) {
    if (G.t == 0) atomicCAS(s.status, 0, (int)RLXPP_ERR_TIMEOUT);
  } else if (live) {
    if constexpr (Kind == kDrawSumHist) {
      uint64_t* sums = static_cast<uint64_t*>(a.out);
      if (sums) sums[i] = a.accumulate_sums ? sums[i] + out.sum : out.sum;
    }
  }
  tc_teardown(smem, G, !ok, phase, T);  // ends with a CTA barrier: the histograms are complete
  if constexpr (Kind == kDrawSumHist) {
    for (int t = tid; t < 256; t += kTcRows * T) {
      unsigned long long tot = 0;
#pragma unroll
      for (int w = 0; w < 4 * T; ++w) tot += hist_s[w * 256 + t];
      if (tot) atomicAdd(a.hist + t, tot);
    }
  }
}

// ---- the fused sum/histogram draw with the A operand in tensor memory ----------------
// A one-tile CTA keeps its operand rows in TMEM next to the accumulator: 128 columns,
// the fp32 accumulator at columns 0..79, row r of the A operand in lane r at columns
// 80..119 (elements 2i and 2i + 1 of the row in the low and high halves of column
// 80 + i).  Each thread writes its own X there with tcgen05.st (its warp owns its 32
// lanes), so per refill the tensor core reads only the level's 12.8 KB matrix from
// shared memory, and no operand row is written to shared memory at all.
constexpr uint32_t kTmA = kTcN;    // first A column
constexpr uint32_t kTmCols = 128;  // TMEM columns of such a CTA
static_assert(kTmA + kTcK / 2 <= kTmCols, "A operand after the accumulator");

// One thread: the five K = 16 products (A from TMEM, the level's matrix from shared
// memory) into the accumulator, committed to the CTA's mbarrier.
__device__ __forceinline__ void tc_issue_tm(uint32_t taddr, uint32_t b0, uint64_t* bar) {
#pragma unroll
  for (int s = 0; s < kTcK / 16; ++s)
    tc_mma_ta(taddr, taddr + kTmA + 8 * s, smem_desc(b0 + s * 2 * kLBO), s > 0 ? 1u : 0u);
  tc_commit(bar);
}

// The fused draw's epilogue: X = sum_k S_k 2^(8k) mod m from the column bit patterns, D its
// 24 RANLUX numbers (Sec. 2.3) and c its borrow, computed without a branch in the common
// case (the fold's limb 0 does not borrow and its carry stops in limb 8, the top limb is
// not all ones, the conversion's
// quick test decides its quotient and X + q carries no further than limb 7); every other
// case (about 2^-15 of the refills) is redone in one branch by the exact forms.  With no
// branch before them, the byte permutes of D's upper limbs (equal to X's) can be
// scheduled while the conversion's carry chain runs.
__device__ __forceinline__ void tc_epilogue_d(const uint32_t col[72], uint32_t X[kLimbs], uint32_t D[kLimbs],
                                              uint32_t& c) {
  uint32_t Xa[kLimbs], T;
  columns_assemble(col, Xa, T);
  // the fold X + T (2^240 - 1) = X + (T - 1) 2^240 + (2^32 - T) + sum_(0<k<7) 0xFFFFFFFF 2^(32k)
  // + 0xFFFF 2^224 when limb 0 does not borrow (Xa_0 >= T, about all but 2^-17 of the
  // refills): limbs 1..6 then come out unchanged and limb 7 gains T 2^16, so the chain
  // is two limbs long
  const bool b0 = Xa[0] < T;
  X[0] = Xa[0] - T;
#pragma unroll
  for (int k = 1; k < 7; ++k) X[k] = Xa[k];
  X[7] = add_cc(Xa[7], T << 16);
  X[8] = addc_cc(Xa[8], 0u);
  const uint32_t c9 = addc(0u, 0u);  // carry out of limb 8
#pragma unroll
  for (int k = 9; k < kLimbs; ++k) X[k] = Xa[k];
  const uint32_t t15 = sub_cc(__funnelshift_l(X[7], X[8], 16), X[15]);
  const uint32_t t16 = subc_cc(__funnelshift_l(X[8], X[9], 16), X[16]);
  const uint32_t t17 = subc_cc(__funnelshift_l(X[9], X[10], 16), X[17]);
  const uint32_t borrow = subc(0u, 0u) & 1u;
  const uint32_t q0 = __funnelshift_l(X[10], X[11], 16);
  D[0] = add_cc(X[0], q0 - borrow);
#pragma unroll
  for (int k = 1; k < 7; ++k) D[k] = addc_cc(X[k], __funnelshift_l(X[10 + k], X[11 + k], 16));
  D[7] = addc_cc(X[7], X[17] >> 16);
  const uint32_t c8 = addc(0u, 0u);  // carry out of limb 7 of X + q
#pragma unroll
  for (int k = 8; k < kLimbs; ++k) D[k] = X[k];
  c = carry_of(X, D);
  const bool rare = b0 || (c9 | c8) != 0u || X[17] == 0xFFFFFFFFu || (t15 & t16 & t17) == 0xFFFFFFFFu ||
                    (t15 | t16 | t17) == 0u || q0 < borrow;
  if (__builtin_expect(rare, 0)) {
#pragma unroll
    for (int k = 0; k < kLimbs; ++k) X[k] = Xa[k];
    fold_x(X, T);
    to_ranlux(X, D);
    c = carry_of(X, D);
  }
}

// The consumer of the fused draw on this kernel: an exact sum and a 256-bin histogram of
// the top 8 bits of every 48-bit value.  The sums of full blocks come from the tensor
// core: the product that refills a block also sums its bytes by position within a
// 48-bit value (columns 72..77, see k_tc_matrix_d), so a block's values add up to
// sum_r 2^(8r) P_r.  The six column bit patterns 0x3F000000 + P_r are accumulated as
// 32-bit multiply-adds by a run-time 1 (FMA pipe) and flushed into the 64-bit total at
// least every 2^20 blocks, while sum P_r < 2^32 is certain (P_r <= 12 * 255).  Values of
// the head and of the stream's last block are added one by one.  The histogram is
// counted per lane: bin b of lane l is word 32 b + l of the tile's table, so the
// increments of a warp fall in 32 different banks; a bin is one byte permute, its
// address one multiply-add by a run-time 128.
constexpr int64_t kFusedFlush = 1 << 20;  // blocks between flushes of the column sums

struct FusedAcc {
  uint64_t total = 0;          // flushed column sums and single values
  uint32_t t[6] = {0, 0, 0, 0, 0, 0};
  uint32_t hist;               // shared address of this lane's column of the table
  uint32_t one, c128;          // 1 and 128, not known to the compiler
  __device__ __forceinline__ void count(uint32_t bin) {
    uint32_t addr;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(addr) : "r"(bin), "r"(c128), "r"(hist));
    asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
  }
  __device__ __forceinline__ void take(uint64_t v) {
    total += v;
    count((uint32_t)(v >> 40));
  }
  __device__ __forceinline__ void hist_block(const uint32_t D[kLimbs]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      count(__byte_perm(D[3 * q + 1], 0u, 0x4441u));  // bits 40..47 of v_2q: byte 1 of D_3q+1
      count(__byte_perm(D[3 * q + 2], 0u, 0x4443u));  // bits 40..47 of v_2q+1: byte 3 of D_3q+2
    }
  }
  __device__ __forceinline__ void columns(const uint32_t s[6]) {
#pragma unroll
    for (int r = 0; r < 6; ++r) asm("mad.lo.u32 %0, %1, %2, %0;" : "+r"(t[r]) : "r"(s[r]), "r"(one));
  }
  // n blocks' column sums into the total (each column carried the 1/2 bias 0x3F000000)
  __device__ __forceinline__ void flush(uint32_t n) {
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      total += (uint64_t)(t[r] - n * 0x3F000000u) << (8 * r);
      t[r] = 0;
    }
  }
};

// Shared memory of the fused CTA besides its static histogram table: the level's matrix
// and the FusedShared words.  With the 32 KB table, a CTA takes 46 KB, so at most four
// share an SM and their 4 x 128 TMEM columns always fit.
constexpr int kFusedDynSmem = kBRegion + 1024;
constexpr int kFusedThreads = kTcRows + 32;  // four compute warps (one tile) and the issuer warp

// Largest value of v over the CTA's threads (v >= 0), through one shared word.
__device__ __forceinline__ int64_t cta_max(int64_t v, unsigned long long* word) {
  if (threadIdx.x == 0) *word = 0ull;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int64_t u = __shfl_xor_sync(0xFFFFFFFFu, v, o);
    v = u > v ? u : v;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(word, (unsigned long long)v);
  __syncthreads();
  return (int64_t)*word;
}

// D (18 limbs) and its borrow c -> the operand row of k_tc_matrix_d: D's 72 bytes as
// fp16 subnormals, then 2048 and 1 (the bias and correction rows), c, zeros.  Every
// thread of the warp calls it (tcgen05.st is warp-wide).
__device__ __forceinline__ void write_d_tmem(uint32_t lane_taddr, const uint32_t D[kLimbs], uint32_t c) {
  uint32_t w[40];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) {
    w[2 * k] = __byte_perm(D[k], 0u, 0x4140u);
    w[2 * k + 1] = __byte_perm(D[k], 0u, 0x4342u);
  }
  w[36] = 0x3C006800u;
  w[37] = c;
  w[38] = 0u;
  w[39] = 0u;
  tmem_st32(lane_taddr + kTmA, w);
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(lane_taddr + kTmA + 32),
               "r"(w[32]), "r"(w[33]), "r"(w[34]), "r"(w[35]), "r"(w[36]), "r"(w[37]), "r"(w[38]), "r"(w[39])
               : "memory");
}

struct FusedShared {
  uint64_t bar;                 // product completion
  uint32_t taddr;               // TMEM base
  uint32_t abort;               // a wait for the product timed out
  unsigned long long iters;     // refills of the tile (its streams' largest count)
};

// The fused draw (exact sum and 256-bin histogram of every stream's doubles, nothing
// written per value) on one-tile CTAs with the A operand in TMEM.  Same semantics as
// k_draw_tc<kDrawSumHist>.  The operand rows hold each stream's RANLUX numbers D and
// borrow c, and the level's matrix is k_tc_matrix_d's, so a product yields the next LCG
// state X and the byte sums of the block it was given.  The tile refills as many times
// as its longest stream needs (one CTA-wide maximum at the start).  Four compute warps
// (one stream a thread) and an issuer warp: each refill, a compute warp waits for the
// product, reads its accumulator rows, forms X, converts it to D and c and writes them as
// its next operand rows (every thread, so that the warp-wide TMEM accesses stay
// converged; rows of finished streams keep advancing), arrives at barrier 1 without
// waiting there, and counts its block into the histogram and adds the previous block's
// column sums while the next product runs; the issuer warp waits at barrier 1 for the
// four and issues the next product.  So no compute warp carries the issue or waits for
// the others.  A wait that gives up (after about 0.3 s) sets the abort flag: that warp
// arrives and leaves, the issuer warp issues nothing more, the other compute warps then
// give up on the product that does not come, and each reports RLXPP_ERR_TIMEOUT.
// one = 1 (a launch argument).
__global__ void __launch_bounds__(kFusedThreads, 4)
    k_fused_tc(const DrawArgs a, const __half* __restrict__ bimg_d, uint32_t one) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(16) unsigned int hist_s[256 * 32];
  const int tid = threadIdx.x;
  const bool issuer_warp = tid >= kTcRows;  // warp 4: issues the products
  {
    uint4* h4 = reinterpret_cast<uint4*>(hist_s);
    for (int w = tid; w < 256 * 32 / 4; w += kFusedThreads) h4[w] = make_uint4(0u, 0u, 0u, 0u);
  }
  FusedShared* sh = reinterpret_cast<FusedShared*>(smem + kBRegion);
  const __half* bmat = tc_bmat(smem);
  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg_d);
    uint4* dst = reinterpret_cast<uint4*>(tc_bmat(smem));
    for (int w = tid; w < kBBytes / 16; w += kFusedThreads) dst[w] = src[w];
  }
  if (tid == 0) {
    mbar_init(&sh->bar, 1);
    fence_barrier_init();
    sh->abort = 0;
  }
  if (tid < 32) tmem_alloc(&sh->taddr, kTmCols);
  fence_proxy_async_smem();  // the level's matrix -> visible to the tensor core
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = sh->taddr;
  const uint32_t lane_taddr = taddr + ((uint32_t)((tid / 32) * 32) << 16);
  const uint32_t b0 = smem_addr(bmat);

  const StateView& s = a.s;
  const uint64_t i = (uint64_t)blockIdx.x * kTcRows + tid;
  const bool live = !issuer_warp && i < s.n;
  int64_t cnt = 0;
  uint32_t pos = kWords, c = 0, lvl = 0;
  uint32_t D[kLimbs];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) D[k] = 0;
  if (live) {
    cnt = a.counts ? a.counts[i] : a.count_each;
    const uint32_t meta = s.meta[i];
    pos = meta_pos(meta);
    c = meta_carry(meta);
    lvl = meta_level(meta);
    load_state_D(s, i, D);
  }
  FusedAcc acc;
  acc.hist = smem_addr(hist_s) + 4u * (uint32_t)(tid & 31);
  acc.one = one;
  acc.c128 = one << 7;
  int64_t rest = cnt;  // values still to draw
  if (live && cnt > 0 && pos + 2 <= (uint32_t)kWords) {  // head of the current block
    const int64_t room = (kWords - pos) / 2;
    const int64_t hcount = cnt < room ? cnt : room;
#pragma unroll
    for (int w = 0; w + 2 <= kWords; ++w) {
      const int d = w - (int)pos;
      if (d >= 0 && d % 2 == 0 && d / 2 < hcount) acc.take(bits48_at_word(D, w));
    }
    rest -= hcount;
    pos += (uint32_t)(hcount * 2);
  }
  // refills of this stream: full blocks, and a last partial one of `tail` values
  const int64_t nref = live && rest > 0 ? (rest + kDoubles - 1) / kDoubles : 0;
  const uint32_t tail = live ? (uint32_t)(rest % kDoubles) : 0u;
  const int64_t iters = cta_max(nref, &sh->iters);
  if (!issuer_warp) {
    write_d_tmem(lane_taddr, D, c);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  volatile uint32_t* vabort = &sh->abort;
  uint32_t phase = 0, c_fin = c;
  bool ok = true, stored = false;
  if (issuer_warp) {
    // one product now and one after each refill but the last, once all four compute
    // warps have arrived at barrier 1 (their rows written, their accumulator rows read)
    uint32_t issued = 0;
    if (iters > 0) {
      if (tid == kTcRows) tc_issue_tm(taddr, b0, &sh->bar);
      issued = 1;
      for (int64_t r = 0; r + 1 < iters; ++r) {
        asm volatile("bar.sync 1, %0;" ::"n"(kFusedThreads) : "memory");
        tc_fence_after();
        if (*vabort) break;
        if (tid == kTcRows) tc_issue_tm(taddr, b0, &sh->bar);
        ++issued;
      }
    }
    // the last product issued is complete before the tensor memory is released
    if (issued) (void)mbar_wait_bounded(&sh->bar, (issued - 1u) & 1u);
  }
  // refills in chunks of at most kFusedFlush, counted in 32 bits within a chunk
  for (int64_t it0 = 0; !issuer_warp && ok && it0 < iters;) {
    const uint32_t n_in = (uint32_t)(iters - it0 > kFusedFlush ? kFusedFlush : iters - it0);
    const bool more_after = it0 + n_in < iters;
    // this stream's refills in the chunk, the one of its last block, and the first whose
    // product carries a block of this stream already drawn whole (not its first block)
    const int64_t rem_ref = nref - it0;
    const uint32_t n_mine = rem_ref <= 0 ? 0u : (rem_ref >= (int64_t)n_in ? n_in : (uint32_t)rem_ref);
    const uint32_t j_last = rem_ref >= 1 && rem_ref <= (int64_t)n_in ? (uint32_t)(rem_ref - 1) : 0xFFFFFFFFu;
    const uint32_t j_sums = it0 == 0 ? 1u : 0u;
    for (uint32_t j = 0; j < n_in; ++j) {
      bool got = mbar_wait_bounded(&sh->bar, phase);
      got = __all_sync(0xFFFFFFFFu, got);  // the warp stays converged for the TMEM accesses
      uint32_t sums[6] = {0, 0, 0, 0, 0, 0};
      if (got) {
        phase ^= 1u;
        tc_fence_after();
        uint32_t col[80];
        tmem_ld64(lane_taddr, col);
        tmem_ld16(lane_taddr + 64, col + 64);
        tmem_wait_ld();
#pragma unroll
        for (int r = 0; r < 6; ++r) sums[r] = col[72 + r];
        uint32_t X[kLimbs];
        tc_epilogue_d(col, X, D, c);
        __syncwarp();  // reconverged after the rare branch, before the warp-wide store
        write_d_tmem(lane_taddr, D, c);
        tmem_wait_st();
      } else {
        *vabort = 1u;
      }
      // this warp's rows are written and its accumulator rows read out: it arrives at
      // barrier 1 (the issuer warp's, which issues the next product once all four have)
      // and goes on at once; a warp that gave up arrives too and leaves, the others
      // then give up on the product that is not issued
      tc_fence_before();
      if (j + 1 < n_in || more_after) asm volatile("bar.arrive 1, %0;" ::"n"(kFusedThreads) : "memory");
      if (!got) {
        ok = false;
        break;
      }
      if (j < n_mine) {  // while the next product computes
        if (j >= j_sums) acc.columns(sums);  // the previous block of this stream, all of it drawn
        if (j != j_last) {
          acc.hist_block(D);  // its sums arrive with the next product
        } else {
          const uint32_t nv = tail ? tail : (uint32_t)kDoubles;
#pragma unroll
          for (int v = 0; v < kDoubles; ++v)
            if (v < (int)nv) acc.take(bits48(D, v));
          store_state_D(s, i, D);
          c_fin = c;
          stored = true;
        }
      }
    }
    acc.flush(n_mine > j_sums ? n_mine - j_sums : 0u);
    it0 += n_in;
  }
  if (nref > 0) pos = tail ? 2u * tail : (uint32_t)kWords;
  if (live && (ok || stored)) s.meta[i] = meta_pack(pos, c_fin, lvl);
  if (!ok) {  // compute warps leave the loop on their own, so each reports
    if ((tid & 31) == 0) atomicCAS(s.status, 0, (int)RLXPP_ERR_TIMEOUT);
  } else if (live) {
    uint64_t* sums = static_cast<uint64_t*>(a.out);
    if (sums) sums[i] = a.accumulate_sums ? sums[i] + acc.total : acc.total;
  }
  // release TMEM (the issuer warp has seen its last product complete)
  tc_fence_before();
  __syncthreads();  // also: every histogram increment is done
  tc_fence_after();
  if (tid < 32) tmem_dealloc(taddr, kTmCols);
  for (int b = tid; b < 256; b += kFusedThreads) {
    unsigned long long tot = 0;
#pragma unroll 8
    for (int l = 0; l < 32; ++l) tot += hist_s[b * 32 + l];
    if (tot) atomicAdd(a.hist + b, tot);
  }
}

// ---- value-writing draws with the A operand in tensor memory -------------------------
struct ValuesShared {
  uint64_t bar;                 // product completion
  uint32_t taddr;               // TMEM base
  uint32_t abort;               // a wait for the product timed out
  unsigned long long iters;     // refills of the tile
  uint32_t pos0;                // read position of the tile's first stream at entry
  int box_x[3];                 // first column of the block staged in each box
  uint32_t box_pending[3];      // a staged box waits for its store
};
// Shared memory: the level's matrix, the shared words, three [128][96 B] staging boxes;
// 50 KB in all, so that at most four CTAs (4 x 128 TMEM columns) share an SM.
constexpr int kValuesBox = kTcRows * kStageBytes;  // 12 KB
constexpr int kValuesBoxes = 3;
constexpr int kValuesSmem = 50 * 1024;
static_assert(kBRegion + 1024 + kValuesBoxes * kValuesBox <= kValuesSmem, "value draw shared memory");
constexpr int kValuesThreads = kTcRows + 32;  // four compute warps (one tile) and the issuer warp

// Value-writing draws (u24, f32, f64) with one count for every stream and the output as
// a [n][count] tensor (tmap), on one-tile CTAs with the A operand in TMEM.  Same
// semantics as k_draw_tc.  The refill loop is the fused draw's, with the same operand
// rows (the RANLUX numbers D and the borrow c), level matrix (k_tc_matrix_d's) and
// issuer warp: the four compute warps wait for the product, form X, convert it to D and
// c, write them as the next operand row (every thread), arrive at the issuer warp's
// barrier and go on to build their block's values and stage them; the issuer warp issues
// the next product once all four have arrived.  When every live stream of the tile
// starts at the tile's first position (then they move in step), the blocks of a refill
// leave as one TMA tensor store of the [128][96 B] staging box, issued by the issuer warp
// at the arrival after the one that follows the staging (thread 0 records the box's
// column in shared memory: it is live whenever any thread is); three boxes rotate.
// Tiles out of step write each stream's values from registers.
template <int Kind>
__global__ void __launch_bounds__(kValuesThreads, 4)
    k_values_tc(const DrawArgs a, const __half* __restrict__ bimg_d, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x;
  const bool issuer_warp = tid >= kTcRows;  // warp 4: issues the products and the stores
  ValuesShared* sh = reinterpret_cast<ValuesShared*>(smem + kBRegion);
  unsigned char* box0 = smem + kBRegion + 1024;
  const __half* bmat = tc_bmat(smem);
  {
    const uint4* src = reinterpret_cast<const uint4*>(bimg_d);
    uint4* dst = reinterpret_cast<uint4*>(tc_bmat(smem));
    for (int w = tid; w < kBBytes / 16; w += kValuesThreads) dst[w] = src[w];
  }
  if (tid == 0) {
    mbar_init(&sh->bar, 1);
    fence_barrier_init();
    sh->abort = 0;
    for (int b = 0; b < kValuesBoxes; ++b) sh->box_pending[b] = 0u;
  }
  if (tid < 32) tmem_alloc(&sh->taddr, kTmCols);
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = sh->taddr;
  const uint32_t lane_taddr = taddr + ((uint32_t)((tid / 32) * 32) << 16);
  const uint32_t b0 = smem_addr(bmat);

  constexpr int need = (Kind == kDrawU24 || Kind == kDrawF32) ? 1 : 2;
  constexpr int per_block = kWords / need;
  const StateView& s = a.s;
  const uint64_t i = (uint64_t)blockIdx.x * kTcRows + tid;
  const bool live = !issuer_warp && i < s.n;
  const int64_t cnt = live ? a.count_each : 0, base = (int64_t)i * a.count_each;
  uint32_t pos = kWords, c = 0, lvl = 0;
  uint32_t D[kLimbs];
#pragma unroll
  for (int k = 0; k < kLimbs; ++k) D[k] = 0;
  if (live) {
    const uint32_t meta = s.meta[i];
    pos = meta_pos(meta);
    c = meta_carry(meta);
    lvl = meta_level(meta);
    load_state_D(s, i, D);
  }
  Consumer<Kind> out;
  out.out = static_cast<decltype(out.out)>(a.out);
  const uint32_t pos_in = pos;
  int64_t k = 0;
  if (live && cnt > 0 && pos + need <= (uint32_t)kWords) {  // head of the current block
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
  // tile-wide stores when every live stream starts at the tile's first position (with
  // one count for all they then stay in step) and the first column after the head is
  // 16-byte aligned; thread 0 (live whenever any thread is) records each staged box
  if (tid == 0) sh->pos0 = pos_in;
  __syncthreads();
  const bool tma =
      __syncthreads_and(!live || (pos_in == sh->pos0 && ((k * (int64_t)(need * 4)) & 15) == 0)) != 0;
  // this stream's refills: full blocks, and a last one of `tail` values (0: full)
  const int64_t nref = live && k < cnt ? (cnt - k + per_block - 1) / per_block : 0;
  const uint32_t tail = (uint32_t)((cnt - k) % per_block);
  const int64_t iters = cta_max(nref, &sh->iters);
  const int y0 = (int)((uint64_t)blockIdx.x * kTcRows);
  if (!issuer_warp) {
    write_d_tmem(lane_taddr, D, c);
    tmem_wait_st();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  volatile uint32_t* vabort = &sh->abort;
  volatile uint32_t* vpend = sh->box_pending;
  volatile int* vbox_x = sh->box_x;
  uint32_t phase = 0, c_fin = c;
  bool ok = true, stored = false;
  if (issuer_warp) {
    // One product now and one after each refill but the last, once the four compute
    // warps have arrived at barrier 1 (their rows written, their accumulator rows read,
    // and the block of the previous refill staged): then also the tile-wide store of
    // that block's box.  Box b is written again two refills after its store is issued,
    // after the product issued at the next arrival; that product waits until the store
    // has read the box.
    const bool lead = tid == kTcRows;
    uint32_t issued = 0;
    if (iters > 0) {
      if (lead) tc_issue_tm(taddr, b0, &sh->bar);
      issued = 1;
      uint32_t box = 0;  // box staged in refill r (r mod 3)
      for (int64_t r = 0; r + 1 < iters; ++r) {
        asm volatile("bar.sync 1, %0;" ::"n"(kValuesThreads) : "memory");
        tc_fence_after();
        if (*vabort) break;
        if (lead) {
          if (tma) bulk_wait_read_all();  // the store issued at the last arrival has read its box
          tc_issue_tm(taddr, b0, &sh->bar);
          const uint32_t pb = box == 0 ? kValuesBoxes - 1 : box - 1;  // staged in refill r - 1
          if (tma && vpend[pb]) {
            vpend[pb] = 0u;
            asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                             reinterpret_cast<uint64_t>(&tmap)),
                         "r"(vbox_x[pb]), "r"(y0), "r"(smem_addr(box0 + pb * kValuesBox))
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
        }
        ++issued;
        box = box == kValuesBoxes - 1 ? 0u : box + 1u;
      }
    }
    if (issued) (void)mbar_wait_bounded(&sh->bar, (issued - 1u) & 1u);
  }
  uint32_t box = 0;  // this refill's staging box (the refill's index mod 3)
  // refills in chunks of at most 2^20, counted in 32 bits within a chunk
  for (int64_t it0 = 0; !issuer_warp && ok && it0 < iters;) {
    const uint32_t n_in = (uint32_t)(iters - it0 > kFusedFlush ? kFusedFlush : iters - it0);
    const bool more_after = it0 + n_in < iters;
    const int64_t rem_ref = nref - it0;
    const uint32_t n_mine = rem_ref <= 0 ? 0u : (rem_ref >= (int64_t)n_in ? n_in : (uint32_t)rem_ref);
    const uint32_t j_last = rem_ref >= 1 && rem_ref <= (int64_t)n_in ? (uint32_t)(rem_ref - 1) : 0xFFFFFFFFu;
    const int64_t k_chunk = k + it0 * per_block;  // this stream's first value of the chunk
    for (uint32_t j = 0; j < n_in; ++j) {
      bool got = mbar_wait_bounded(&sh->bar, phase);
      got = __all_sync(0xFFFFFFFFu, got);  // the warp stays converged for the TMEM accesses
      if (got) {
        phase ^= 1u;
        tc_fence_after();
        uint32_t col[72];
        tmem_ld64(lane_taddr, col);
        tmem_ld8(lane_taddr + 64, col + 64);
        tmem_wait_ld();
        uint32_t X[kLimbs];
        tc_epilogue_d(col, X, D, c);
        __syncwarp();  // reconverged after the rare branch, before the warp-wide store
        write_d_tmem(lane_taddr, D, c);
        tmem_wait_st();
      } else {
        *vabort = 1u;
      }
      // this warp's rows are written and its accumulator rows read out: it arrives at
      // the issuer warp's barrier and goes on at once; a warp that gave up arrives too
      // and leaves, the others then give up on the product that is not issued
      tc_fence_before();
      if (j + 1 < n_in || more_after) asm volatile("bar.arrive 1, %0;" ::"n"(kValuesThreads) : "memory");
      if (!got) {
        ok = false;
        break;
      }
      if (j < n_mine) {  // this stream's block, while the next product computes
        const int64_t kj = k_chunk + (int64_t)j * per_block;
        const bool full = j != j_last || tail == 0;
        if (tma) {  // the whole block into this thread's row of the box; past the count it is clipped
          uint4 v[6];
          block_values<Kind>(D, v);
          uint4* rowp = reinterpret_cast<uint4*>(box0 + box * kValuesBox + tid * kStageBytes);
#pragma unroll
          for (int q = 0; q < 6; ++q) rowp[q] = v[q];
          fence_proxy_async_smem();
          if (tid == 0) {
            vbox_x[box] = (int)kj;
            vpend[box] = 1u;
          }
        } else if (full) {
          out.block(D, base + kj);
        } else {
          out.partial(D, base + kj, tail);
        }
        if (j == j_last) {
          c_fin = c;
          store_state_D(s, i, D);
          stored = true;
        }
      }
      box = box == kValuesBoxes - 1 ? 0u : box + 1u;
    }
    it0 += n_in;
  }
  if (nref > 0) {
    k = cnt;
    pos = tail ? tail * need : (uint32_t)kWords;
  }
  if (live && (ok || stored)) s.meta[i] = meta_pack(pos, c_fin, lvl);
  if (!ok && (tid & 31) == 0) atomicCAS(s.status, 0, (int)RLXPP_ERR_TIMEOUT);
  // every block is staged: the boxes the loop did not store (those of the last two
  // refills) leave now, and the CTA ends once every store is done
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == kTcRows && tma && !*vabort) {
#pragma unroll 1
    for (int64_t r = iters - 2; r < iters; ++r) {
      if (r < 0) continue;
      const uint32_t pb = (uint32_t)(r % kValuesBoxes);
      if (vpend[pb]) {
        vpend[pb] = 0u;
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                         reinterpret_cast<uint64_t>(&tmap)),
                     "r"(vbox_x[pb]), "r"(y0), "r"(smem_addr(box0 + pb * kValuesBox))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
  }
  if (tid == kTcRows) bulk_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(taddr, kTmCols);
}

constexpr int kReqThreads = kTcRows + 32;  // four compute warps (one tile) and the issuer warp

// Emits the unread part of the current block for a value kind (f64 or u24).
__device__ __forceinline__ void emit_head(bool f64, const BatchArgs& b, const uint32_t D[kLimbs], uint32_t& pos,
                                          int64_t cnt, int64_t base, int64_t& k) {
  const int need = f64 ? 2 : 1;
  if (cnt <= 0 || pos + need > (uint32_t)kWords) return;
  const int64_t room = (kWords - pos) / need;
  const int64_t h = cnt < room ? cnt : room;
#pragma unroll
  for (int w = 0; w < kWords; ++w) {
    const int d = w - (int)pos;
    if (d < 0 || d % need != 0 || d / need >= h) continue;
    if (f64) {
      if (w + 1 < kWords) b.out_f64[base + d / 2] = f64_bits_from48_outlined(bits48_at_word(D, w));
    } else {
      b.out_u24[base + d] = word24(D, w);
    }
  }
  k = h;
  pos += (uint32_t)(h * need);
}

// Batched requests on the tensor cores, every luxury level in one launch.  Persistent
// one-tile CTAs take tiles from the counter: a tile is up to 128 consecutive chunks of
// one level of the (per level, longest-first) list, and the tile table itself is
// ordered longest first across levels.  A CTA loads the level's matrix into shared
// memory when it changes from the previous tile's; then every thread jumps its chunk to
// its start block (table products on the integer pipe) and the tile refills in lock step
// with the fused draw's pipelined loop (operand rows in TMEM, one barrier per refill,
// the next product issued before the blocks are converted and written) until its
// longest chunk is done.  Chunks of a tile have similar lengths, so little work is lost
// to the longest one.  Plain chunks write to unrelated places: each lane stages its full
// block, and the warp writes its 32 staged blocks cooperatively.  A strided tile (up to
// four warps of 32 strided chunks, kItemStrided) multiplies by the level's A^32, so each
// lane steps 32 blocks a refill and a warp's 32 blocks of one refill are consecutive in
// the output: the warp writes them as one contiguous run (warp_store_run).
__global__ void __launch_bounds__(kReqThreads, 4)
    k_requests_tc(const BatchArgs b, const Item* __restrict__ items, const TcTile* __restrict__ tiles,
                  uint64_t n_tiles, const __half* __restrict__ bimg_all, const __half* __restrict__ bimg32_all,
                  WorkCounters* wc) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ unsigned long long tile_s;
  const int tid = threadIdx.x;
  const bool issuer_warp = tid >= kTcRows;  // warp 4: issues the products
  ValuesShared* sh = reinterpret_cast<ValuesShared*>(smem + kBRegion);
  unsigned char* stage = smem + kBRegion + 1024;
  uint4* slot = reinterpret_cast<uint4*>(stage + tid * kStageBytes);
  const unsigned char* wstage = stage + (tid & ~31) * kStageBytes;  // this warp's 32 slots
  const __half* bmat = tc_bmat(smem);
  if (tid == 0) {
    mbar_init(&sh->bar, 1);
    fence_barrier_init();
    sh->abort = 0;
  }
  if (tid < 32) tmem_alloc(&sh->taddr, kTmCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = sh->taddr;
  const uint32_t lane_taddr = taddr + ((uint32_t)((tid / 32) * 32) << 16);
  const uint32_t b0 = smem_addr(bmat);
  volatile uint32_t* vabort = &sh->abort;
  uint32_t phase = 0, issued = 0;  // issued: products issued (the issuer warp's count)
  bool ok = true;
  uint32_t loaded = 0xFFFFFFFFu;  // level whose matrix is in shared memory
  while (ok) {
    if (tid == 0) tile_s = atomicAdd(&wc->next, 1ull);
    __syncthreads();
    const unsigned long long t = tile_s;
    __syncthreads();  // every thread has read the tile index
    if (t >= n_tiles) break;
    const TcTile tile = tiles[t];
    const bool strided = (tile.level & kTileStrided) != 0;  // the tile's chunks step by A^32
    if (tile.level != loaded) {  // the products of the previous tile are complete
      const uint4* src = reinterpret_cast<const uint4*>((strided ? bimg32_all : bimg_all) +
                                                        (size_t)(tile.level & ~kTileStrided) * (kBBytes / 2));
      uint4* dst = reinterpret_cast<uint4*>(tc_bmat(smem));
      for (int w = tid; w < kBBytes / 16; w += kReqThreads) dst[w] = src[w];
      fence_proxy_async_smem();  // -> visible to the tensor core after the next barrier
      loaded = tile.level;
    }
    const bool live = (uint32_t)tid < tile.n;
    Item it{};
    if (live) it = items[tile.first + tid];
    uint32_t D[kLimbs];
#pragma unroll
    for (int q = 0; q < kLimbs; ++q) D[q] = 0;
    uint32_t c = 0, lvl = 0;
    if (live) {
      uint32_t meta;
      request_state(b, it.req, D, meta);
      lvl = meta_level(meta);
      c = meta_carry(meta);
      if (it.jump) {  // X <- A^jump X
        uint32_t X[kLimbs];
        to_lcg(D, c, X);
        bool have = true;
        apply_digits(b.s.table + (size_t)lvl * kTableLimbs, 0, it.jump, X, have);
        to_ranlux(X, D);
        c = carry_of(X, D);
      }
    }
    const bool f64 = (it.info & 1u) != 0;
    const int64_t cnt = live ? it.count : 0, base = (int64_t)it.out;
    // a strided chunk's next block is kStride blocks on: the values drawn so far (k, whole
    // blocks) stand for kStride as many places in the output
    const int64_t ostep = strided ? (int64_t)kStride : 1;
    const int64_t per = f64 ? kDoubles : kWords;
    uint32_t pos = live ? (it.info >> 8) & 0xFFu : (uint32_t)kWords;
    int64_t k = 0;
    emit_head(f64, b, D, pos, cnt, base, k);
    int64_t left = live && k < cnt ? (cnt - k + per - 1) / per : 0;
    const int64_t iters = cta_max(left, &sh->iters);
    // the stream's state after the request's last chunk (written when its last block is
    // drawn, since the operand rows of a finished chunk keep advancing)
    const bool final_state = live && b.advance && ((it.info >> 16) & 1u);
    const uint64_t st = final_state ? b.req_stream[it.req] : 0;
    if (final_state && left == 0) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        b.s.D[(uint64_t)q * b.s.stride + st] = ((uint64_t)D[2 * q + 1] << 32) | D[2 * q];
      b.s.meta[st] = meta_pack(pos, c, lvl);
    }
    if (!issuer_warp) {
      write_d_tmem(lane_taddr, D, c);
      tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (issuer_warp && iters > 0) {
      // one product now and one after each refill but the last, once the four compute
      // warps have arrived at barrier 1 (their rows written, their accumulator rows read)
      if (tid == kTcRows) tc_issue_tm(taddr, b0, &sh->bar);
      ++issued;
      for (int64_t r = 0; r + 1 < iters; ++r) {
        asm volatile("bar.sync 1, %0;" ::"n"(kReqThreads) : "memory");
        tc_fence_after();
        if (*vabort) break;
        if (tid == kTcRows) tc_issue_tm(taddr, b0, &sh->bar);
        ++issued;
      }
    }
    for (int64_t r = 0; !issuer_warp && r < iters; ++r) {
      bool got = mbar_wait_bounded(&sh->bar, phase);
      got = __all_sync(0xFFFFFFFFu, got);  // the warp stays converged for the TMEM accesses
      if (got) {
        phase ^= 1u;
        tc_fence_after();
        uint32_t col[72];
        tmem_ld64(lane_taddr, col);
        tmem_ld8(lane_taddr + 64, col + 64);
        tmem_wait_ld();
        uint32_t X[kLimbs];
        tc_epilogue_d(col, X, D, c);
        __syncwarp();  // reconverged after the rare branch, before the warp-wide store
        write_d_tmem(lane_taddr, D, c);
        tmem_wait_st();
      } else {
        *vabort = 1u;
      }
      // this warp's rows are written and its accumulator rows read out: it arrives at
      // the issuer warp's barrier and goes on at once; a warp that gave up arrives too
      // and leaves, the others then give up on the product that is not issued
      tc_fence_before();
      if (r + 1 < iters) asm volatile("bar.arrive 1, %0;" ::"n"(kReqThreads) : "memory");
      if (!got) {
        ok = false;
        break;
      }
      uint64_t dst = 0;  // destination of this lane's full block, if it has one
      if (left > 0) {    // this chunk's block, while the next product computes
        const int64_t rem = cnt - k;
        if (rem >= per) {
          uint4 v[6];
          if (f64)
            block_values<kDrawF64>(D, v);
          else
            block_values<kDrawU24>(D, v);
#pragma unroll
          for (int q = 0; q < 6; ++q) slot[q] = v[q];
          dst = f64 ? reinterpret_cast<uint64_t>(b.out_f64 + base + ostep * k)
                    : reinterpret_cast<uint64_t>(b.out_u24 + base + ostep * k);
          k += per;
          pos = kWords;
        } else {
          if (f64) {
#pragma unroll
            for (int j = 0; j < kDoubles; ++j)
              if (j < rem) b.out_f64[base + ostep * k + j] = f64_bits_from48_outlined(bits48(D, j));
            pos = (uint32_t)(rem * 2);
          } else {
#pragma unroll
            for (int j = 0; j < kWords; ++j)
              if (j < rem) b.out_u24[base + ostep * k + j] = word24(D, j);
            pos = (uint32_t)rem;
          }
          k = cnt;
        }
        if (--left == 0 && final_state) {
#pragma unroll
          for (int q = 0; q < 9; ++q)
            b.s.D[(uint64_t)q * b.s.stride + st] = ((uint64_t)D[2 * q + 1] << 32) | D[2 * q];
          b.s.meta[st] = meta_pack(pos, c, lvl);
        }
      }
      if (strided)
        warp_store_run(wstage, dst);
      else
        warp_store_blocks(wstage, dst);
    }
    // every warp has left the tile's loop (on a timeout, after its own wait ran out):
    // the CTA goes on to the next tile together, or stops together
    if (issuer_warp && *vabort) ok = false;
    ok = __syncthreads_and(ok) != 0;
  }
  if (!ok && tid == 0) atomicCAS(b.s.status, 0, (int)RLXPP_ERR_TIMEOUT);
  // the last product issued is complete before the tensor memory is released
  if (issuer_warp && issued) (void)mbar_wait_bounded(&sh->bar, (issued - 1u) & 1u);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid < 32) tmem_dealloc(taddr, kTmCols);
  finish_cta(wc);
}

// One tensor-path product per item: out = A x mod m (x < m), for testing.  With
// issue == 0 no MMA is issued, so the barrier never completes and the bounded wait
// must give up and report RLXPP_ERR_TIMEOUT.
__global__ void __launch_bounds__(kTcRows, 4) k_tc_mulmod(const __half* __restrict__ bimg, const uint64_t* x,
                                                          uint64_t* out, uint64_t n, int* status, int issue) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const TcGroup G = tc_group(smem, false);  // one group per CTA
  tc_setup(smem, G, bimg, 1);
  const uint32_t taddr = tc_tmem(smem, G);
  const uint64_t i = (uint64_t)blockIdx.x * kTcRows + threadIdx.x;
  uint32_t X[kLimbs];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const uint64_t v = i < n ? x[9 * i + k] : 0;
    X[2 * k] = (uint32_t)v;
    X[2 * k + 1] = (uint32_t)(v >> 32);
  }
  write_x_row(G.tile, G.t, X);
  uint32_t col[72], phase = 0;
  const bool ok = tc_refill(G, tc_bmat(smem), taddr, phase, col, issue != 0);
  if (ok) {
    columns_to_x(col, X);
    if (i < n)
#pragma unroll
      for (int k = 0; k < 9; ++k) out[9 * i + k] = ((uint64_t)X[2 * k + 1] << 32) | X[2 * k];
  } else if (threadIdx.x == 0) {
    atomicCAS(status, 0, (int)RLXPP_ERR_TIMEOUT);
  }
  tc_teardown(smem, G, !ok && issue, phase, 1);  // nothing is in flight when no MMA was issued
}

// The level's matrix in the shared-memory image layout: column j (K index) holds the
// bytes of R_j = A 2^(8j) mod m for j < 72, 2^-12 for j = 72 (against 2048: the 1/2
// bias), the bytes of E as fp16 subnormals e_k 2^-24 for j = 73, zeros after.
__global__ void k_tc_matrix(const uint32_t* __restrict__ lux, __half* __restrict__ bimg) {
  const int j = threadIdx.x;  // 0..79
  if (j >= kTcK) return;
  uint8_t bytes[kTcN];
  if (j < 72) {
    uint32_t P[2 * kLimbs];
#pragma unroll 1
    for (int q = 0; q < 2 * kLimbs; ++q) P[q] = 0;
    const int sh_limb = (8 * j) >> 5, sh_bit = (8 * j) & 31;
#pragma unroll 1
    for (int q = 0; q < kLimbs; ++q) {
      const uint32_t a = lux[q];
      P[q + sh_limb] |= a << sh_bit;
      if (sh_bit) P[q + sh_limb + 1] |= a >> (32 - sh_bit);
    }
    uint32_t R[kLimbs];
    mod_m(P, R);
#pragma unroll 1
    for (int n = 0; n < kTcN; ++n) bytes[n] = n < 72 ? (uint8_t)(R[n >> 2] >> (8 * (n & 3))) : 0;
  } else if (j == 73) {
    // E = -C mod m, C = 0x3F003F000000 sum_{t<18} 2^(32t): limbs 0x3F000000, then
    // 0x3F003F00 (limbs 1..17) and 0x3F00 (limb 18)
    uint32_t P[2 * kLimbs];
#pragma unroll 1
    for (int q = 0; q < 2 * kLimbs; ++q) P[q] = q == 0 ? 0x3F000000u : (q < kLimbs ? 0x3F003F00u : 0u);
    P[kLimbs] = 0x3F00u;
    uint32_t R[kLimbs], E[kLimbs];
    mod_m(P, R);
    // E = m - R (R != 0 here; m = 2^576 - 2^240 + 1)
    uint64_t borrow = 0;
#pragma unroll 1
    for (int q = 0; q < kLimbs; ++q) {
      const uint32_t mq = q == 0 ? 1u : (q < 7 ? 0u : (q == 7 ? 0xFFFF0000u : 0xFFFFFFFFu));
      const uint64_t d = (uint64_t)mq - R[q] - borrow;
      E[q] = (uint32_t)d;
      borrow = (d >> 63) & 1u;
    }
#pragma unroll 1
    for (int n = 0; n < kTcN; ++n) bytes[n] = n < 72 ? (uint8_t)(E[n >> 2] >> (8 * (n & 3))) : 0;
  }
#pragma unroll 1
  for (int n = 0; n < kTcN; ++n) {
    // level bytes as integers; 2^-12 (x 2048 = 1/2) for the bias row; e_k 2^-24 (exact
    // fp16 subnormals) for the correction row
    const float v = j < 72 ? (float)bytes[n]
                           : (j == 72 ? 0x1p-12f : (j == 73 ? (float)bytes[n] * 0x1p-24f : 0.f));
    bimg[tc_off(n, j)] = __float2half(v);
  }
}

// The level's matrix for products whose operand rows hold a stream's RANLUX numbers D
// and borrow c instead of its LCG state (the fused draw).  X = D - floor(D / 2^336) + c
// is linear in the 72 bytes d_j of D: byte j stands for 2^(8j), less 2^(8j - 336) for
// j >= 42, so A X = sum_j d_j R'_j + c A (mod m) with R'_j = A 2^(8j) - A 2^(8(j-42)) =
// R_j - R_(j-42) mod m for j >= 42 and R'_j = R_j below.  Column k < 72 of row j holds
// byte k of R'_j; row 74 holds the bytes of A (against c); rows 72 and 73 are the bias
// and correction rows of k_tc_matrix.  Columns 72..77 of row j < 72 hold 1 when j mod 6
// equals the column's index r = k - 72, so that those columns sum the bytes of D by
// their position within a 48-bit value: the 48-bit values of the block add up to
// sum_r 2^(8r) P_r, P_r the sum in column 72 + r (below 12 * 255).
__device__ __forceinline__ void lux_shift_mod(const uint32_t* __restrict__ lux, int j, uint32_t R[kLimbs]) {
  uint32_t P[2 * kLimbs];
#pragma unroll 1
  for (int q = 0; q < 2 * kLimbs; ++q) P[q] = 0;
  const int sh_limb = (8 * j) >> 5, sh_bit = (8 * j) & 31;
#pragma unroll 1
  for (int q = 0; q < kLimbs; ++q) {
    const uint32_t a = lux[q];
    P[q + sh_limb] |= a << sh_bit;
    if (sh_bit) P[q + sh_limb + 1] |= a >> (32 - sh_bit);
  }
  mod_m(P, R);
}

__global__ void k_tc_matrix_d(const uint32_t* __restrict__ lux, __half* __restrict__ bimg) {
  const int j = threadIdx.x;  // 0..79
  if (j >= kTcK) return;
  float v[kTcN];
#pragma unroll 1
  for (int n = 0; n < kTcN; ++n) v[n] = 0.f;
  if (j < 72) {
    uint32_t R[kLimbs];
    lux_shift_mod(lux, j, R);
    if (j >= 42) {  // R - R_(j-42) mod m (both in [0, m))
      uint32_t S[kLimbs];
      lux_shift_mod(lux, j - 42, S);
      uint64_t borrow = 0;
#pragma unroll 1
      for (int q = 0; q < kLimbs; ++q) {
        const uint64_t d = (uint64_t)R[q] - S[q] - borrow;
        R[q] = (uint32_t)d;
        borrow = (d >> 63) & 1u;
      }
      if (borrow) {  // + m = 2^576 - 2^240 + 1 (the wrap past 2^576 cancels the borrow)
        uint64_t carry = 0;
#pragma unroll 1
        for (int q = 0; q < kLimbs; ++q) {
          const uint32_t mq = q == 0 ? 1u : (q < 7 ? 0u : (q == 7 ? 0xFFFF0000u : 0xFFFFFFFFu));
          const uint64_t t = (uint64_t)R[q] + mq + carry;
          R[q] = (uint32_t)t;
          carry = t >> 32;
        }
      }
    }
#pragma unroll 1
    for (int n = 0; n < 72; ++n) v[n] = (float)((R[n >> 2] >> (8 * (n & 3))) & 0xFFu);
    v[72 + j % 6] = 1.f;
  } else if (j == 72) {  // against 2048: 1/2 in every column
#pragma unroll 1
    for (int n = 0; n < kTcN; ++n) v[n] = 0x1p-12f;
  } else if (j == 73) {  // against 1: the bytes of E = -C mod m as subnormals
    uint32_t P[2 * kLimbs];
#pragma unroll 1
    for (int q = 0; q < 2 * kLimbs; ++q) P[q] = q == 0 ? 0x3F000000u : (q < kLimbs ? 0x3F003F00u : 0u);
    P[kLimbs] = 0x3F00u;
    uint32_t R[kLimbs], E[kLimbs];
    mod_m(P, R);
    uint64_t borrow = 0;
#pragma unroll 1
    for (int q = 0; q < kLimbs; ++q) {
      const uint32_t mq = q == 0 ? 1u : (q < 7 ? 0u : (q == 7 ? 0xFFFF0000u : 0xFFFFFFFFu));
      const uint64_t d = (uint64_t)mq - R[q] - borrow;
      E[q] = (uint32_t)d;
      borrow = (d >> 63) & 1u;
    }
#pragma unroll 1
    for (int n = 0; n < 72; ++n) v[n] = (float)((E[n >> 2] >> (8 * (n & 3))) & 0xFFu) * 0x1p-24f;
  } else if (j == 74) {  // against the borrow c: the bytes of A
#pragma unroll 1
    for (int n = 0; n < 72; ++n) v[n] = (float)((lux[n >> 2] >> (8 * (n & 3))) & 0xFFu);
  }
#pragma unroll 1
  for (int n = 0; n < kTcN; ++n) bimg[tc_off(n, j)] = __float2half(v[n]);
}

// One-group CTAs (the request and test kernels, the fused and Gaussian draws) take
// 48 KB of dynamic shared memory, so that at most 4 share an SM, whose 512 TMEM columns
// then always suffice; the value-writing draws run kTcGroups groups per CTA and one CTA
// per SM.  (Five groups per CTA made the fused draw slower: its per-warp shared-memory
// histogram took about twice the bank-conflicted atomic wavefronts.)
constexpr size_t kTcSmem = 48 * 1024;
static_assert(tc_smem_bytes(1, true) <= (int)kTcSmem, "shared memory layout");
constexpr int kTcGroups = 5;
static_assert(tc_smem_bytes(kTcGroups, true) <= 227 * 1024, "shared memory of a five-group CTA");
// Tile-groups per CTA of each draw kernel.
template <int Kind>
constexpr int tc_groups() {
  return (Kind == kDrawSumHist || Kind == kDrawNormal || Kind == kDrawExp) ? 1 : kTcGroups;
}

// cuTensorMapEncodeTiled from the driver, looked up once (null if unavailable).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The output of a draw with one count for every stream as a [n][count_each] tensor with a
// [128][per block] box, when the TMA can address it: 16-byte aligned base and row
// stride, and coordinates within 32 bits.  Returns false otherwise (the kernel then
// writes each stream's blocks by itself).
template <int Kind>
bool encode_output_map(const DrawArgs& a, CUtensorMap* map) {
  constexpr uint64_t esize = Kind == kDrawF64 ? 8 : 4;
  constexpr uint32_t per_block = Kind == kDrawF64 ? kDoubles : kWords;
  if (a.counts != nullptr || a.count_each <= 0 || a.s.n == 0) return false;
  const uint64_t cols = (uint64_t)a.count_each, rows = a.s.n;
  if (cols > 0x7FFFFFFFull || rows > 0x7FFFFFFFull) return false;
  if ((reinterpret_cast<uintptr_t>(a.out) & 15) != 0 || ((cols * esize) & 15) != 0) return false;
  if (cols * esize >= (1ull << 40)) return false;
  const EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {cols * esize};
  const cuuint32_t box[2] = {per_block, (cuuint32_t)kTcRows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, esize == 8 ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, a.out,
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int Kind>
cudaError_t launch_tc_kind(const DrawArgs& a, const __half* bimg, const __half* bimg_d, cudaStream_t st) {
  constexpr int T = tc_groups<Kind>();
  // one-group CTAs keep 48 KB so that at most 4 share an SM (512 TMEM columns)
  constexpr int smem_bytes = T == 1 ? (int)kTcSmem : tc_smem_bytes(T, Kind != kDrawSumHist);
  constexpr bool kValues = Kind == kDrawU24 || Kind == kDrawF64 || Kind == kDrawF32;
  const uint64_t tiles = (a.s.n + kTcRows - 1) / kTcRows;
  const unsigned grid = (unsigned)((tiles + T - 1) / T);
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  int use_tma = 0;
  if constexpr (kValues) use_tma = encode_output_map<Kind>(a, &map) ? 1 : 0;
  if constexpr (kValues) {
    if (use_tma) {  // one count for all and a tensor map: one-tile CTAs, A operand in TMEM
      cudaError_t e = cudaFuncSetAttribute(k_values_tc<Kind>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kValuesSmem);
      if (e != cudaSuccess) return e;
      k_values_tc<Kind><<<(unsigned)tiles, kValuesThreads, kValuesSmem, st>>>(a, bimg_d, map);
      return cudaGetLastError();
    }
  }
  auto kern = (kValues && !use_tma) ? k_draw_tc<Kind, T, kValues> : k_draw_tc<Kind, T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, kTcRows * T, smem_bytes, st>>>(a, bimg, map, use_tma);
  return cudaGetLastError();
}

cudaError_t launch_fused_tc(const DrawArgs& a, const __half* bimg_d, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_fused_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kFusedDynSmem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((a.s.n + kTcRows - 1) / kTcRows);
  k_fused_tc<<<grid, kFusedThreads, kFusedDynSmem, st>>>(a, bimg_d, 1u);
  return cudaGetLastError();
}

}  // namespace

size_t tc_matrix_bytes() { return kBBytes; }

cudaError_t launch_requests_tc(const BatchArgs& b, const Item* items, const TcTile* tiles, uint64_t n_tiles,
                               const void* bimg, const void* bimg32, WorkCounters* wc, unsigned grid,
                               cudaStream_t st) {
  if (n_tiles == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_requests_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  if (grid > n_tiles) grid = (unsigned)n_tiles;
  k_requests_tc<<<grid, kReqThreads, kTcSmem, st>>>(b, items, tiles, n_tiles, static_cast<const __half*>(bimg),
                                                    static_cast<const __half*>(bimg32), wc);
  return cudaGetLastError();
}

cudaError_t launch_tc_matrix(const uint32_t* lux18, void* bimg, cudaStream_t st) {
  k_tc_matrix<<<1, kTcK, 0, st>>>(lux18, static_cast<__half*>(bimg));
  return cudaGetLastError();
}

cudaError_t launch_tc_matrix_d(const uint32_t* lux18, void* bimg, cudaStream_t st) {
  k_tc_matrix_d<<<1, kTcK, 0, st>>>(lux18, static_cast<__half*>(bimg));
  return cudaGetLastError();
}

cudaError_t launch_draw_tc(int kind, const DrawArgs& a, const void* bimg, const void* bimg_d, cudaStream_t st) {
  if (a.s.n == 0) return cudaSuccess;
  const __half* b = static_cast<const __half*>(bimg);
  const __half* bd = static_cast<const __half*>(bimg_d);
  switch (kind) {
    case kDrawU24: return launch_tc_kind<kDrawU24>(a, b, bd, st);
    case kDrawF64: return launch_tc_kind<kDrawF64>(a, b, bd, st);
    case kDrawSumHist: return launch_fused_tc(a, bd, st);
    case kDrawF32: return launch_tc_kind<kDrawF32>(a, b, bd, st);
    case kDrawNormal: return launch_tc_kind<kDrawNormal>(a, b, bd, st);
    case kDrawExp: return launch_tc_kind<kDrawExp>(a, b, bd, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_mulmod(const void* bimg, const uint64_t* x, uint64_t* out, uint64_t n, int* status,
                             cudaStream_t st, bool issue) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_tc_mulmod, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (e != cudaSuccess) return e;
  k_tc_mulmod<<<(unsigned)((n + kTcRows - 1) / kTcRows), kTcRows, kTcSmem, st>>>(static_cast<const __half*>(bimg),
                                                                                 x, out, n, status, issue ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace rlxpp
