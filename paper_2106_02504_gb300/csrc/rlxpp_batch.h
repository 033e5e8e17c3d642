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
  uint32_t info;    // bit 0: kind (1 = f64); bits 8..15: read position; bit 16: last chunk
};

struct BatchArgs {
  const uint64_t* req_stream;  // [n_reqs]
  uint64_t* snap_D;            // [9][n_reqs]
  uint32_t* snap_meta;         // [n_reqs]
  uint64_t n_reqs;
  StateView s;                 // resident states (final states are written back here)
  uint32_t* out_u24;
  uint64_t* out_f64;
  int advance;
};

// Tensor-core request kernel: items[0..n) of one luxury level whose matrix is bimg.
cudaError_t launch_requests_tc(const BatchArgs& b, const Item* items, uint64_t n, const void* bimg,
                               cudaStream_t st);

}  // namespace rlxpp
