// Internal declarations shared by the translation units of librlxpp.so.
#pragma once
#include <cstddef>
#include <cstdint>
#include <map>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/rlxpp.h"

namespace rlxpp {

// Power table for skips and seeds (Sec. 2.4): entry (w, j) = A^(j 16^w) mod m for
// windows w < kWindows (exponents below 2^160 = 2^96 * 2^64 seeds) and digits j < 16
// (j = 0 unused), each 18 limbs of 32 bits.
constexpr int kWindows = 40;
constexpr int kDigits = 16;
constexpr size_t kTableLimbs = (size_t)kWindows * kDigits * 18;
constexpr int kSeedWindow0 = 24;  // 2^96 = 16^24

// Resident per-stream state, structure of arrays:
//   D      9 planes of n uint64 (plane k holds bits 64k..64k+63 of every stream's D);
//   meta   n uint32: bits 0..7 read position (0..24), bit 8 borrow, bits 16..23 level.
__host__ __device__ inline uint32_t meta_pack(uint32_t pos, uint32_t carry, uint32_t level) {
  return pos | (carry << 8) | (level << 16);
}
__host__ __device__ inline uint32_t meta_pos(uint32_t m) { return m & 0xFFu; }
__host__ __device__ inline uint32_t meta_carry(uint32_t m) { return (m >> 8) & 1u; }
__host__ __device__ inline uint32_t meta_level(uint32_t m) { return (m >> 16) & 0xFFu; }

struct Lux {  // a luxury multiplier in kernel-parameter (constant bank) form
  uint32_t a[18];   // A, 32-bit limbs
  uint32_t as[9];   // A0 + A1 mod 2^288 (A = A1 2^288 + A0), for the Karatsuba product
  uint32_t ca;      // carry of A0 + A1
};

struct StateView {
  uint64_t* D;       // [9][stride], this view's streams first
  uint32_t* meta;    // [n]
  uint64_t n;        // streams in this view
  uint64_t stride;   // distance between the planes of D (streams of the handle)
  const uint32_t* lux;    // [n_levels][18] multipliers A
  const uint32_t* table;  // [n_levels][kTableLimbs]
  int* status;       // sticky device status (rlxpp_status value, 0 = ok)
};

enum DrawKind {
  kDrawU24 = 0,
  kDrawF64 = 1,
  kDrawSumHist = 2,
  kDrawF32 = 3,
  kDrawNormal = 4,
  kDrawExp = 5,
  kDrawRaw52 = 6  // raw LCG doubles, 11 per refill (integer path only)
};

struct DrawArgs {
  StateView s;
  Lux A;                 // used when `uniform` (every stream at level 0)
  int uniform;
  const int64_t* counts;   // NULL: count_each for all, out offset i * count_each
  const int64_t* offsets;
  int64_t count_each;
  void* out;             // uint32 / double output, or per-stream sums (sum/hist)
  unsigned long long* hist;  // 256 bins (sum/hist)
  int accumulate_sums;   // sum/hist: add to sums[i] instead of overwriting
};

constexpr int kDrawBlock = 128;  // threads per block of the draw kernels

// ---- kernels launchers (defined in the .cu files) --------------------------------
cudaError_t launch_level_setup(uint32_t p, uint32_t* lux_out18, uint32_t* table_out,
                               cudaStream_t st);
// keep_levels: take each stream's level from its current meta word (re-seeding)
cudaError_t launch_seed(const StateView& s, const uint64_t* seeds, const uint8_t* level_of_stream,
                        uint32_t n_levels, bool keep_levels, cudaStream_t st);
cudaError_t launch_skip(const StateView& s, const uint64_t* n128, cudaStream_t st);
// move each stream as if n[i] values of `need` numbers each had been drawn
cudaError_t launch_skip_values(const StateView& s, const uint64_t* n, uint32_t need, cudaStream_t st);
cudaError_t launch_draw(int kind, const DrawArgs& a, cudaStream_t st);
// one warp per stream (RLXPP_PATH_WARP); warp_draw_supported: the kinds it has
bool warp_draw_supported(int kind);
cudaError_t launch_draw_warp(int kind, const DrawArgs& a, cudaStream_t st);
cudaError_t launch_export(const StateView& s, const uint32_t* level_p, rlxpp_state* dst,
                          cudaStream_t st);
cudaError_t launch_import(const StateView& s, const uint32_t* level_p, uint32_t n_levels,
                          const rlxpp_state* src, cudaStream_t st);
// tensor-core refill (rlxpp_tensor.cu)
size_t tc_matrix_bytes();
cudaError_t launch_tc_matrix(const uint32_t* lux18, void* bimg, cudaStream_t st);
// the matrix for operand rows that hold (D, c) instead of X, with the block-sum columns
cudaError_t launch_tc_matrix_d(const uint32_t* lux18, void* bimg, cudaStream_t st);
cudaError_t launch_draw_tc(int kind, const DrawArgs& a, const void* bimg, const void* bimg_d, cudaStream_t st);
cudaError_t launch_tc_mulmod(const void* bimg, const uint64_t* x, uint64_t* out, uint64_t n, int* status,
                             cudaStream_t st, bool issue = true);
// True when rlxpp_test_fail_alloc asked for this device allocation to fail (the caller
// then reports cudaErrorMemoryAllocation without allocating).
bool injected_alloc_failure();

// Warp-arithmetic unit tests (rlxpp_warp.cu): op 0 mod_m of 18-uint64 inputs, op 1 the
// conversion to RANLUX numbers of 9-uint64 states (with carry).
cudaError_t launch_warp_test(int op, const uint64_t* in, uint64_t* out, uint32_t* carry, uint64_t n,
                             cudaStream_t st);

cudaError_t launch_test(int which, const uint64_t* x, const uint64_t* y, uint64_t* out,
                        uint32_t* carry, uint64_t n, cudaStream_t st);

enum TestOp {
  kTestMultiply = 0,
  kTestModM = 1,
  kTestMulMod = 2,
  kTestToRanlux = 3,
  kTestToLcg = 4,
  kTestF64 = 5,
  kTestNegLn48 = 6,
  kTestCosSin2Pi48 = 7,
  kTestBoxMuller48 = 8
};

// Records msg as the calling thread's rlxpp_last_error() text and returns code.
rlxpp_status set_last_error(rlxpp_status code, const char* msg);

// Reads the request tuner's saved choices for this device model (RLXPP_TUNE_CACHE).
void load_tune_cache(rlxpp_gen* g);

}  // namespace rlxpp

// The handle behind rlxpp_gen* (opaque in the public header).
struct rlxpp_gen {
  int device = 0;
  uint64_t n = 0;
  uint32_t n_levels = 0;
  uint32_t levels[RLXPP_MAX_LEVELS] = {};
  rlxpp::Lux lux_host[RLXPP_MAX_LEVELS] = {};
  uint64_t* D = nullptr;        // [9][n]
  uint32_t* meta = nullptr;     // [n]
  uint32_t* lux = nullptr;      // [n_levels][18]
  uint32_t* table = nullptr;    // [n_levels][kTableLimbs]
  uint32_t* level_p = nullptr;  // [n_levels]
  int* status = nullptr;        // sticky device status
  cudaStream_t copy_stream = nullptr;  // device-to-host copies of chunked host output
  cudaEvent_t ev[4] = {};
  void* host_stage = nullptr;          // device staging of the asynchronous host draws
  size_t host_stage_bytes = 0;
  cudaEvent_t chunk_ready = nullptr;   // a staged chunk is complete (compute stream)
  cudaEvent_t host_done = nullptr;     // the last asynchronous host draw's copies are done
  int sms = 0;                         // multiprocessors of the device
  std::map<uint32_t, rlxpp_tuning> tuned;  // request-shape signature -> tuner choice
  std::vector<uint8_t> level_host;         // host copy of every stream's level index
  bool level_host_stale = false;           // set_state may have changed levels
  uint32_t path = 0;                       // RLXPP_PATH_IMAD or RLXPP_PATH_TENSOR
  void* tc_matrix = nullptr;               // [n_levels] tensor-path matrices
  void* tc_matrix_d = nullptr;             // [n_levels] the same for (D, c) operand rows
  void* tc_matrix_d32 = nullptr;           // [n_levels] the same for the multiplier A^32 (strided chunks)
  struct Upload {                          // page-locked staging of request work lists
    void* host = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;              // its last copies are done
  };
  Upload upload[2];
  int upload_next = 0;
  rlxpp::StateView view() const { return rlxpp::StateView{D, meta, n, n, lux, table, status}; }
};

