// Work items of batched requests, shared by the integer-pipe and tensor-core request
// kernels.
#pragma once
#include <cstdint>

#include "rlxpp_internal.h"

namespace rlxpp {

struct Item {       // one chunk (32 bytes)
  uint64_t jump;    // LCG advances from the request's start state to this chunk's block
  int64_t count;    // values
  uint64_t out;     // index of the first value in the output array of its kind
  uint32_t req;     // request index
  uint32_t info;    // bit 0: kind (1 = f64); bits 8..15: read position; bit 16: last chunk;
                    // bit 17: strided (its blocks are 32 apart, see kItemStrided)
};
// A strided chunk (tensor path) is one lane of a warp of 32 chunks of one request: lane t
// draws blocks f + t, f + t + 32, f + t + 64, ... (one product by A^32 per refill), so the
// warp's 32 blocks of a refill are consecutive in the output and leave as one contiguous
// run.  Its first block is reached by its jump and drawn from read position 0; the j-th
// block after it goes to out + 32 j per.
constexpr uint32_t kItemStrided = 1u << 17;
constexpr uint32_t kStride = 32;             // blocks between a strided chunk's blocks
constexpr uint32_t kTileStrided = 1u << 31;  // TcTile::level flag: the tile's items are strided
constexpr uint32_t kTcTileWarps = 4;         // warps of a tensor-path tile (128 rows)

struct BatchArgs {
  const uint64_t* req_stream;  // [n_reqs]
  uint64_t* snap_D;            // [9][n_reqs], or null: read the resident state directly
  uint32_t* snap_meta;         // [n_reqs]
  uint64_t n_reqs;
  StateView s;                 // resident states (final states are written back here)
  uint32_t* out_u24;
  uint64_t* out_f64;
  int advance;
};

// One tile of the tensor-core request kernel: up to 128 consecutive items of one luxury
// level (items[first .. first + n)); a strided tile (level | kTileStrided) holds up to four
// warps of 32 strided chunks each and multiplies by the level's A^32.
struct TcTile {
  uint64_t first;
  uint32_t n;
  uint32_t level;
};

// Work counters of a persistent request kernel: [0] the next item or tile to take,
// [1] CTAs that have finished.  Zero before a launch; the last CTA to finish sets both
// back to zero, so that the next launch (a replayed graph included) needs no reset.
struct WorkCounters {
  unsigned long long next, done;
};

#ifdef __CUDACC__
// The state (24 numbers as 18 limbs, and the meta word) of request r's stream at the
// start of the run: from the snapshot when the run writes states back (the final state
// of a stream must not change what its other chunks read), else the resident state.
__device__ __forceinline__ void request_state(const BatchArgs& b, uint32_t r, uint32_t D[18], uint32_t& meta) {
  if (b.snap_D) {
    meta = b.snap_meta[r];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const uint64_t v = b.snap_D[(uint64_t)q * b.n_reqs + r];
      D[2 * q] = (uint32_t)v;
      D[2 * q + 1] = (uint32_t)(v >> 32);
    }
  } else {
    const uint64_t st = b.req_stream[r];
    meta = b.s.meta[st];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const uint64_t v = b.s.D[(uint64_t)q * b.s.stride + st];
      D[2 * q] = (uint32_t)v;
      D[2 * q + 1] = (uint32_t)(v >> 32);
    }
  }
}

// End of a CTA of a persistent request kernel (after its last use of the counters):
// the last one to finish resets them.
__device__ __forceinline__ void finish_cta(WorkCounters* wc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&wc->done, 1ull) == (unsigned long long)(gridDim.x - 1)) {
      wc->next = 0ull;
      wc->done = 0ull;
    }
  }
}
#endif

// Tensor-core request kernel: persistent CTAs over the tile table, every level in one
// launch; bimg holds the levels' matrices one after the other.
cudaError_t launch_requests_tc(const BatchArgs& b, const Item* items, const TcTile* tiles, uint64_t n_tiles,
                               const void* bimg, const void* bimg32, WorkCounters* wc, unsigned grid,
                               cudaStream_t st);
// Warp-cooperative request kernel (one warp per chunk; rlxpp_warp.cu): every level in one
// launch, the level's multiplier read from the state view's table; tpb threads per CTA
// (64, 128 or 256).
cudaError_t launch_requests_warp(const BatchArgs& b, const Item* items, uint64_t n_items, WorkCounters* wc,
                                 unsigned grid, uint32_t tpb, cudaStream_t st);

// Threads per CTA of a tuning (0: the default, 128).
inline uint32_t tuning_tpb(const rlxpp_tuning& t) { return t.threads_per_block ? t.threads_per_block : 128u; }

}  // namespace rlxpp
