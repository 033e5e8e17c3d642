// Host side of the C ABI declared in include/rlxpp.h: argument checks, device memory
// of the generator state, staging of host buffers, and the launches.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rlxpp_internal.h"

using namespace rlxpp;

namespace {

thread_local std::string g_last_error;

// Host logging to stderr, chosen once by the environment variable RLXPP_LOG: 0 (or
// unset) silent, 1 every failed call with its message, 2 also each create, destroy,
// draw, skip and seed call with its main arguments.
int log_level() {
  static const int level = [] {
    const char* v = std::getenv("RLXPP_LOG");
    return v ? std::atoi(v) : 0;
  }();
  return level;
}

rlxpp_status fail(rlxpp_status code, const std::string& msg) {
  g_last_error = msg;
  if (log_level() >= 1) std::fprintf(stderr, "rlxpp: error %d: %s\n", (int)code, msg.c_str());
  return code;
}

#define RLX_LOG_CALL(...)                          \
  do {                                             \
    if (log_level() >= 2) {                        \
      std::fprintf(stderr, "rlxpp: " __VA_ARGS__); \
      std::fputc('\n', stderr);                    \
    }                                              \
  } while (0)

std::atomic<int64_t> g_fail_alloc{-1};  // rlxpp_test_fail_alloc's countdown (-1: off)

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (injected_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, st);
}
template <class T>
cudaError_t dev_malloc_async(T** p, size_t bytes, cudaStream_t st) {
  return dev_malloc_async(reinterpret_cast<void**>(p), bytes, st);
}

// The status of a failed CUDA call: out of device memory is RLXPP_ERR_NOMEM.
rlxpp_status cuda_status(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? RLXPP_ERR_NOMEM : RLXPP_ERR_CUDA;
}

#define RLX_CUDA(expr)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (expr);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      return fail(cuda_status(e_), std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    }                                                                                   \
  } while (0)

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Where a pointer lives, seen from the current device: memory the current device can
// dereference directly (its own device memory, or managed memory), host memory (also
// unregistered), or device memory of another GPU, which the kernels must not be given
// (without peer access the first load would fault).
enum class Mem { kHost, kDevice, kOtherDevice };
Mem mem_kind(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return Mem::kHost;
  }
  if (attr.type == cudaMemoryTypeManaged) return Mem::kDevice;
  if (attr.type != cudaMemoryTypeDevice) return Mem::kHost;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return Mem::kOtherDevice;
  }
  return attr.device == cur ? Mem::kDevice : Mem::kOtherDevice;
}
bool on_device(const void* p) { return mem_kind(p) == Mem::kDevice; }

// Seeds start at 1.  A host array is checked here (the call then fails at once); zeros
// in a device array are reported by the seeding kernel (sticky RLXPP_ERR_INVALID).
bool host_seeds_valid(const uint64_t* seeds, uint64_t n) {
  if (on_device(seeds)) return true;
  for (uint64_t i = 0; i < n; ++i)
    if (seeds[i] == 0) return false;
  return true;
}

// A device copy of a host input array, or the pointer itself if already on the device.
// The copy completes before this returns, so the caller's host buffer may be reused.
struct Staged {
  void* dev = nullptr;
  bool owned = false;
  cudaStream_t st = nullptr;
  ~Staged() {
    if (owned && dev) cudaFreeAsync(dev, st);
  }
};

rlxpp_status stage_in(const void* src, size_t bytes, cudaStream_t st, Staged& out) {
  out.st = st;
  if (src != nullptr && mem_kind(src) == Mem::kOtherDevice)
    return fail(RLXPP_ERR_INVALID, "an input array is device memory of another GPU");
  if (src == nullptr || bytes == 0 || on_device(src)) {
    out.dev = const_cast<void*>(src);
    return RLXPP_OK;
  }
  RLX_CUDA(dev_malloc_async(&out.dev, bytes, st));
  out.owned = true;
  RLX_CUDA(cudaMemcpyAsync(out.dev, src, bytes, cudaMemcpyHostToDevice, st));
  RLX_CUDA(cudaStreamSynchronize(st));
  return RLXPP_OK;
}

rlxpp_status check_gen(const rlxpp_gen* g) {
  if (!g) return fail(RLXPP_ERR_INVALID, "null generator handle");
  RLX_CUDA(cudaSetDevice(g->device));
  return RLXPP_OK;
}

rlxpp_status setup_levels(rlxpp_gen* g, cudaStream_t st) {
  for (uint32_t l = 0; l < g->n_levels; ++l) {
    cudaError_t e = launch_level_setup(g->levels[l], g->lux + (size_t)l * 18,
                                       g->table + (size_t)l * kTableLimbs, st);
    if (e != cudaSuccess) return fail(cuda_status(e), std::string("level setup: ") + cudaGetErrorString(e));
  }
  std::vector<uint32_t> limbs(18 * g->n_levels);
  RLX_CUDA(cudaMemcpyAsync(limbs.data(), g->lux, sizeof(uint32_t) * limbs.size(), cudaMemcpyDeviceToHost, st));
  RLX_CUDA(cudaStreamSynchronize(st));
  for (uint32_t l = 0; l < g->n_levels; ++l) {  // kernel-parameter form of each multiplier
    Lux& x = g->lux_host[l];
    std::memcpy(x.a, limbs.data() + 18 * l, sizeof x.a);
    uint64_t carry = 0;
    for (int k = 0; k < 9; ++k) {
      const uint64_t t = (uint64_t)x.a[k] + x.a[9 + k] + carry;
      x.as[k] = (uint32_t)t;
      carry = t >> 32;
    }
    x.ca = (uint32_t)carry;
  }
  return RLXPP_OK;
}

void free_gen(rlxpp_gen* g) {
  if (!g) return;
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  cudaFree(g->D);
  cudaFree(g->meta);
  cudaFree(g->lux);
  cudaFree(g->table);
  cudaFree(g->level_p);
  cudaFree(g->status);
  cudaFree(g->tc_matrix);
  cudaFree(g->tc_matrix_d);
  cudaFree(g->tc_matrix_d32);
  for (auto& u : g->upload) {
    if (u.ev) cudaEventDestroy(u.ev);
    if (u.host) cudaFreeHost(u.host);
  }
  cudaFree(g->host_stage);
  if (g->chunk_ready) cudaEventDestroy(g->chunk_ready);
  if (g->host_done) cudaEventDestroy(g->host_done);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  delete g;
}

DrawArgs make_args(const rlxpp_gen* g) {
  DrawArgs a{};
  a.s = g->view();
  a.uniform = g->n_levels == 1;
  a.A = g->lux_host[0];
  return a;
}

constexpr size_t kChunkBytes = size_t(256) << 20;  // device staging per chunk of host output

// The draw kernels of the handle's path: tensor cores when the handle has one luxury
// level (a tile's streams share the multiplier matrix), one warp per stream for the
// kinds the warp kernel has, else the integer pipe.
cudaError_t launch_path(const rlxpp_gen* g, int kind, const DrawArgs& a, cudaStream_t st) {
  if (kind == kDrawRaw52) return launch_draw(kind, a, st);  // integer pipe only
  if (g->path == RLXPP_PATH_TENSOR && g->n_levels == 1)
    return launch_draw_tc(kind, a, g->tc_matrix, g->tc_matrix_d, st);
  if (g->path == RLXPP_PATH_WARP && warp_draw_supported(kind)) return launch_draw_warp(kind, a, st);
  return launch_draw(kind, a, st);
}

// Draw of kind (u24 / f64) into out; host outputs go through device chunks that are
// copied back on a second stream while the next chunk computes.
rlxpp_status draw_common(rlxpp_gen* g, int kind, const int64_t* counts, const int64_t* offsets,
                         int64_t count_each, void* out, size_t elem, cudaStream_t st) {
  RLX_LOG_CALL("draw kind %d gen %p count_each %lld per-stream counts %s out %p", kind, (void*)g,
               (long long)count_each, counts ? "yes" : "no", out);
  if (rlxpp_status s = check_gen(g)) return s;
  if (g->n == 0) return RLXPP_OK;
  if (!counts && count_each < 0) return fail(RLXPP_ERR_INVALID, "count_each must be >= 0");
  if (counts && !offsets) return fail(RLXPP_ERR_INVALID, "offsets required with counts");
  if (!out) {
    if (!counts && count_each == 0) return RLXPP_OK;
    return fail(RLXPP_ERR_INVALID, "null output");
  }
  if (mem_kind(out) == Mem::kOtherDevice) return fail(RLXPP_ERR_INVALID, "output is device memory of another GPU");
  Staged sc, so;
  if (rlxpp_status s = stage_in(counts, sizeof(int64_t) * g->n, st, sc)) return s;
  if (rlxpp_status s = stage_in(offsets, sizeof(int64_t) * g->n, st, so)) return s;
  DrawArgs a = make_args(g);
  a.counts = static_cast<const int64_t*>(sc.dev);
  a.offsets = static_cast<const int64_t*>(so.dev);
  a.count_each = count_each;
  if (on_device(out)) {
    a.out = out;
    cudaError_t e = launch_path(g, kind, a, st);
    if (e != cudaSuccess) return fail(cuda_status(e), std::string("draw: ") + cudaGetErrorString(e));
    return RLXPP_OK;
  }
  if (counts) {
    // host output with per-stream ranges: one device image of the whole output
    std::vector<int64_t> hc(g->n), ho(g->n);
    RLX_CUDA(cudaMemcpyAsync(hc.data(), a.counts, sizeof(int64_t) * g->n, cudaMemcpyDeviceToHost, st));
    RLX_CUDA(cudaMemcpyAsync(ho.data(), a.offsets, sizeof(int64_t) * g->n, cudaMemcpyDeviceToHost, st));
    RLX_CUDA(cudaStreamSynchronize(st));
    int64_t total = 0;
    for (uint64_t i = 0; i < g->n; ++i) {
      if (hc[i] < 0 || ho[i] < 0) return fail(RLXPP_ERR_INVALID, "negative count or offset");
      if (hc[i] > 0) total = std::max(total, ho[i] + hc[i]);
    }
    if (total == 0) return RLXPP_OK;
    void* dev = nullptr;
    RLX_CUDA(dev_malloc_async(&dev, (size_t)total * elem, st));
    // keep untouched elements of the caller's buffer: start from its contents
    cudaError_t e = cudaMemcpyAsync(dev, out, (size_t)total * elem, cudaMemcpyHostToDevice, st);
    a.out = dev;
    if (e == cudaSuccess) e = launch_path(g, kind, a, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, dev, (size_t)total * elem, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(dev, st);
    if (e != cudaSuccess) return fail(cuda_status(e), std::string("draw to host: ") + cudaGetErrorString(e));
    return RLXPP_OK;
  }
  if (count_each == 0) return RLXPP_OK;
  // uniform counts: chunks of whole streams, double-buffered (one buffer when a second
  // cannot be had)
  const size_t per_stream = (size_t)count_each * elem;
  uint64_t chunk = std::max<uint64_t>(1, kChunkBytes / per_stream);
  chunk = std::min<uint64_t>(chunk, g->n);
  void* buf[2] = {nullptr, nullptr};
  RLX_CUDA(dev_malloc_async(&buf[0], chunk * per_stream, st));
  cudaError_t e = dev_malloc_async(&buf[1], chunk * per_stream, st);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    buf[1] = nullptr;
    e = cudaSuccess;
  }
  const int nbuf = buf[1] ? 2 : 1;
  int k = 0;
  for (uint64_t s0 = 0; e == cudaSuccess && s0 < g->n; s0 += chunk, ++k) {
    const uint64_t s1 = std::min<uint64_t>(g->n, s0 + chunk);
    const int b = k % nbuf;
    if (k >= nbuf) e = cudaStreamWaitEvent(st, g->ev[2 + b], 0);  // buffer b copied out
    if (e != cudaSuccess) break;
    DrawArgs c = a;
    c.s.D = g->D + s0;  // a view of streams s0..s1-1 (plane stride stays n)
    c.s.meta = g->meta + s0;
    c.s.n = s1 - s0;
    c.out = buf[b];
    e = launch_path(g, kind, c, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev[b], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->copy_stream, g->ev[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(out) + s0 * per_stream, buf[b], (s1 - s0) * per_stream,
                          cudaMemcpyDeviceToHost, g->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev[2 + b], g->copy_stream);
  }
  cudaError_t e2 = cudaStreamSynchronize(g->copy_stream);
  if (e == cudaSuccess) e = e2;
  cudaStreamWaitEvent(st, g->ev[2], 0);
  if (nbuf == 2) cudaStreamWaitEvent(st, g->ev[3], 0);
  cudaFreeAsync(buf[0], st);
  if (buf[1]) cudaFreeAsync(buf[1], st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail(cuda_status(e), std::string("draw to host: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

// Asynchronous draw of count_each values per stream into page-locked host memory:
// chunks of whole streams are computed on st into the handle's staging buffer and each
// is copied out on the copy stream behind an event; nothing waits on the host.
rlxpp_status draw_host_async(rlxpp_gen* g, int kind, int64_t count_each, void* out, size_t elem,
                             cudaStream_t st) {
  RLX_LOG_CALL("draw to host (asynchronous) kind %d gen %p count_each %lld out %p", kind, (void*)g,
               (long long)count_each, out);
  if (rlxpp_status s = check_gen(g)) return s;
  if (count_each < 0) return fail(RLXPP_ERR_INVALID, "count_each must be >= 0");
  if (g->n == 0 || count_each == 0) return RLXPP_OK;
  if (!out) return fail(RLXPP_ERR_INVALID, "null output");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, out) != cudaSuccess || attr.type != cudaMemoryTypeHost) {
    cudaGetLastError();
    return fail(RLXPP_ERR_INVALID, "asynchronous host draws need page-locked host memory");
  }
  const size_t per_stream = (size_t)count_each * elem;
  const size_t total = per_stream * g->n;
  // the staging buffer is free again once the previous asynchronous draw's copies are done
  RLX_CUDA(cudaStreamWaitEvent(st, g->host_done, 0));
  if (g->host_stage_bytes < total) {
    cudaFree(g->host_stage);  // waits for the device, copies of the old buffer included
    g->host_stage = nullptr;
    g->host_stage_bytes = 0;
    RLX_CUDA(dev_malloc(&g->host_stage, total));
    g->host_stage_bytes = total;
  }
  DrawArgs a = make_args(g);
  a.count_each = count_each;
  const uint64_t chunk = std::min<uint64_t>(g->n, std::max<uint64_t>(1, kChunkBytes / per_stream));
  cudaError_t e = cudaSuccess;
  for (uint64_t s0 = 0; e == cudaSuccess && s0 < g->n; s0 += chunk) {
    const uint64_t s1 = std::min<uint64_t>(g->n, s0 + chunk);
    DrawArgs c = a;
    c.s.D = g->D + s0;  // a view of streams s0..s1-1 (plane stride stays n)
    c.s.meta = g->meta + s0;
    c.s.n = s1 - s0;
    c.out = static_cast<char*>(g->host_stage) + s0 * per_stream;
    e = launch_path(g, kind, c, st);
    if (e == cudaSuccess) e = cudaEventRecord(g->chunk_ready, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->copy_stream, g->chunk_ready, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(out) + s0 * per_stream, c.out, (s1 - s0) * per_stream,
                          cudaMemcpyDeviceToHost, g->copy_stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(g->host_done, g->copy_stream);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("draw to host (asynchronous): ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

}  // namespace

// Failure injection for the tests (rlxpp_test_fail_alloc): the device allocation that
// brings the countdown to zero reports cudaErrorMemoryAllocation without allocating.
bool rlxpp::injected_alloc_failure() {
  int64_t c = g_fail_alloc.load();
  while (c >= 0) {
    if (g_fail_alloc.compare_exchange_weak(c, c - 1)) return c == 0;
  }
  return false;
}

rlxpp_status rlxpp::set_last_error(rlxpp_status code, const char* msg) {
  return fail(code, msg);
}

extern "C" {

rlxpp_status rlxpp_create(uint64_t n_streams, const uint32_t* levels, uint32_t n_levels,
                          const uint8_t* level_of_stream, const uint64_t* seeds,
                          void* cuda_stream, rlxpp_gen** out) {
  RLX_LOG_CALL("create %llu streams, %u levels (first p %u)", (unsigned long long)n_streams, n_levels,
               levels && n_levels ? levels[0] : 0u);
  if (!out) return fail(RLXPP_ERR_INVALID, "null output handle pointer");
  *out = nullptr;
  if (!levels || n_levels == 0 || n_levels > RLXPP_MAX_LEVELS)
    return fail(RLXPP_ERR_INVALID, "need 1..RLXPP_MAX_LEVELS luxury levels");
  for (uint32_t l = 0; l < n_levels; ++l)
    if (levels[l] == 0) return fail(RLXPP_ERR_INVALID, "luxury level must be >= 1");
  if (n_streams > 0 && !seeds) return fail(RLXPP_ERR_INVALID, "null seeds");
  if (n_streams > (uint64_t(1) << 40)) return fail(RLXPP_ERR_INVALID, "too many streams");
  if (n_streams > 0 && !host_seeds_valid(seeds, n_streams)) return fail(RLXPP_ERR_INVALID, "seeds must be >= 1");
  cudaStream_t st = as_stream(cuda_stream);
  rlxpp_gen* g = new rlxpp_gen();
  auto bail = [&](rlxpp_status s) {
    free_gen(g);
    return s;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess) return bail(fail(RLXPP_ERR_CUDA, "no CUDA device"));
  if (cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return bail(fail(RLXPP_ERR_CUDA, "cannot read the multiprocessor count"));
  load_tune_cache(g);
  g->n = n_streams;
  g->n_levels = n_levels;
  std::memcpy(g->levels, levels, sizeof(uint32_t) * n_levels);
  const size_t nn = std::max<uint64_t>(n_streams, 1);
  cudaError_t e = dev_malloc(&g->D, sizeof(uint64_t) * 9 * nn);
  if (e == cudaSuccess) e = dev_malloc(&g->meta, sizeof(uint32_t) * nn);
  if (e == cudaSuccess) e = dev_malloc(&g->lux, sizeof(uint32_t) * 18 * n_levels);
  if (e == cudaSuccess) e = dev_malloc(&g->table, sizeof(uint32_t) * kTableLimbs * n_levels);
  if (e == cudaSuccess) e = dev_malloc(&g->level_p, sizeof(uint32_t) * n_levels);
  if (e == cudaSuccess) e = dev_malloc(&g->status, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking);
  for (auto& ev : g->ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->chunk_ready, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->host_done, cudaEventDisableTiming);
  if (e != cudaSuccess)
    return bail(fail(cuda_status(e), std::string("create: ") + cudaGetErrorString(e)));
  e = cudaMemsetAsync(g->status, 0, sizeof(int), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g->level_p, g->levels, sizeof(uint32_t) * n_levels, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->D, 0, sizeof(uint64_t) * 9 * nn, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->meta, 0, sizeof(uint32_t) * nn, st);
  if (e != cudaSuccess) return bail(fail(cuda_status(e), std::string("create: ") + cudaGetErrorString(e)));
  if (rlxpp_status s = setup_levels(g, st)) return bail(s);
  {  // tensor-path matrices of every level; the tensor path is the default
    e = dev_malloc(&g->tc_matrix, tc_matrix_bytes() * n_levels);
    if (e == cudaSuccess) e = dev_malloc(&g->tc_matrix_d, tc_matrix_bytes() * n_levels);
    if (e == cudaSuccess) e = dev_malloc(&g->tc_matrix_d32, tc_matrix_bytes() * n_levels);
    for (uint32_t l = 0; e == cudaSuccess && l < n_levels; ++l) {
      e = launch_tc_matrix(g->lux + (size_t)l * 18, static_cast<char*>(g->tc_matrix) + tc_matrix_bytes() * l, st);
      if (e == cudaSuccess)
        e = launch_tc_matrix_d(g->lux + (size_t)l * 18, static_cast<char*>(g->tc_matrix_d) + tc_matrix_bytes() * l,
                               st);
      // A^32 = power-table entry (window 1, digit 2): the multiplier of strided request chunks
      if (e == cudaSuccess)
        e = launch_tc_matrix_d(g->table + (size_t)l * kTableLimbs + (size_t)(1 * kDigits + 2) * 18,
                               static_cast<char*>(g->tc_matrix_d32) + tc_matrix_bytes() * l, st);
    }
    if (e != cudaSuccess) return bail(fail(cuda_status(e), std::string("tensor setup: ") + cudaGetErrorString(e)));
    g->path = RLXPP_PATH_TENSOR;
  }
  if (n_streams > 0) {
    Staged ss, sl;
    if (rlxpp_status s = stage_in(seeds, sizeof(uint64_t) * n_streams, st, ss)) return bail(s);
    if (rlxpp_status s = stage_in(level_of_stream, n_streams, st, sl)) return bail(s);
    e = launch_seed(g->view(), static_cast<const uint64_t*>(ss.dev), static_cast<const uint8_t*>(sl.dev),
                    n_levels, false, st);
    if (e != cudaSuccess) return bail(fail(cuda_status(e), std::string("seed: ") + cudaGetErrorString(e)));
    g->level_host.assign(n_streams, 0);
    if (sl.dev) {  // host copy of the level indices (out-of-range ones were seeded at level 0)
      e = cudaMemcpyAsync(g->level_host.data(), sl.dev, n_streams, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return bail(fail(cuda_status(e), std::string("levels: ") + cudaGetErrorString(e)));
      for (auto& l : g->level_host)
        if (l >= n_levels) l = 0;
    }
  }
  *out = g;
  return RLXPP_OK;
}

rlxpp_status rlxpp_seed(rlxpp_gen* g, const uint64_t* seeds, void* cuda_stream) {
  RLX_LOG_CALL("seed gen %p", (void*)g);
  if (rlxpp_status s = check_gen(g)) return s;
  if (g->n == 0) return RLXPP_OK;
  if (!seeds) return fail(RLXPP_ERR_INVALID, "null seeds");
  if (!host_seeds_valid(seeds, g->n)) return fail(RLXPP_ERR_INVALID, "seeds must be >= 1");
  cudaStream_t st = as_stream(cuda_stream);
  Staged ss;
  if (rlxpp_status s = stage_in(seeds, sizeof(uint64_t) * g->n, st, ss)) return s;
  cudaError_t e = launch_seed(g->view(), static_cast<const uint64_t*>(ss.dev), nullptr, g->n_levels,
                              true, st);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("seed: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

rlxpp_status rlxpp_skip(rlxpp_gen* g, const uint64_t* n128, void* cuda_stream) {
  RLX_LOG_CALL("skip gen %p", (void*)g);
  if (rlxpp_status s = check_gen(g)) return s;
  if (g->n == 0) return RLXPP_OK;
  if (!n128) return fail(RLXPP_ERR_INVALID, "null skip distances");
  cudaStream_t st = as_stream(cuda_stream);
  Staged sn;
  if (rlxpp_status s = stage_in(n128, sizeof(uint64_t) * 2 * g->n, st, sn)) return s;
  cudaError_t e = launch_skip(g->view(), static_cast<const uint64_t*>(sn.dev), st);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("skip: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

rlxpp_status rlxpp_draw_u24(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, uint32_t* out, void* cuda_stream) {
  return draw_common(g, kDrawU24, counts, offsets, count_each, out, sizeof(uint32_t),
                     as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_f64(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, double* out, void* cuda_stream) {
  return draw_common(g, kDrawF64, counts, offsets, count_each, out, sizeof(double),
                     as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_f32(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, float* out, void* cuda_stream) {
  return draw_common(g, kDrawF32, counts, offsets, count_each, out, sizeof(float), as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_u24_host_async(rlxpp_gen* g, int64_t count_each, uint32_t* out, void* cuda_stream) {
  return draw_host_async(g, kDrawU24, count_each, out, sizeof(uint32_t), as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_f64_host_async(rlxpp_gen* g, int64_t count_each, double* out, void* cuda_stream) {
  return draw_host_async(g, kDrawF64, count_each, out, sizeof(double), as_stream(cuda_stream));
}

rlxpp_status rlxpp_host_wait(rlxpp_gen* g, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  RLX_CUDA(cudaStreamWaitEvent(as_stream(cuda_stream), g->host_done, 0));
  return RLXPP_OK;
}

rlxpp_status rlxpp_draw_normal_f64(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, double* out, void* cuda_stream) {
  return draw_common(g, kDrawNormal, counts, offsets, count_each, out, sizeof(double), as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_exp_f64(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                            int64_t count_each, double* out, void* cuda_stream) {
  return draw_common(g, kDrawExp, counts, offsets, count_each, out, sizeof(double), as_stream(cuda_stream));
}

rlxpp_status rlxpp_draw_raw_f64(rlxpp_gen* g, const int64_t* counts, const int64_t* offsets,
                                int64_t count_each, double* out, void* cuda_stream) {
  return draw_common(g, kDrawRaw52, counts, offsets, count_each, out, sizeof(double), as_stream(cuda_stream));
}

rlxpp_status rlxpp_skip_values(rlxpp_gen* g, const uint64_t* n_values, uint32_t kind, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  if (kind != RLXPP_KIND_U24 && kind != RLXPP_KIND_F64 && kind != RLXPP_KIND_F32)
    return fail(RLXPP_ERR_INVALID, "unknown value kind");
  if (g->n == 0) return RLXPP_OK;
  if (!n_values) return fail(RLXPP_ERR_INVALID, "null counts");
  cudaStream_t st = as_stream(cuda_stream);
  Staged sn;
  if (rlxpp_status s = stage_in(n_values, sizeof(uint64_t) * g->n, st, sn)) return s;
  cudaError_t e = launch_skip_values(g->view(), static_cast<const uint64_t*>(sn.dev),
                                     kind == RLXPP_KIND_F64 ? 2u : 1u, st);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("skip values: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

rlxpp_status rlxpp_draw_f64_sum_hist(rlxpp_gen* g, int64_t count_each, uint64_t* sums,
                                     uint64_t* hist, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  if (count_each < 0) return fail(RLXPP_ERR_INVALID, "count_each must be >= 0");
  if (!hist) return fail(RLXPP_ERR_INVALID, "null histogram");
  if (!on_device(hist) || (sums && !on_device(sums)))
    return fail(RLXPP_ERR_INVALID, "sums and hist must be device memory");
  if (g->n == 0) return RLXPP_OK;
  cudaStream_t st = as_stream(cuda_stream);
  DrawArgs a = make_args(g);
  a.out = sums;
  a.hist = reinterpret_cast<unsigned long long*>(hist);
  // per-warp 32-bit shared-memory bins: at most 2^26 values per lane and launch
  const int64_t kMaxPerLaunch = int64_t(1) << 26;
  int64_t done = 0;
  do {
    a.count_each = std::min(count_each - done, kMaxPerLaunch);
    a.accumulate_sums = done > 0;
    cudaError_t e = launch_path(g, kDrawSumHist, a, st);
    if (e != cudaSuccess) return fail(cuda_status(e), std::string("sum/hist: ") + cudaGetErrorString(e));
    done += a.count_each;
  } while (done < count_each);
  return RLXPP_OK;
}

rlxpp_status rlxpp_get_state(const rlxpp_gen* g, rlxpp_state* dst, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  if (g->n == 0) return RLXPP_OK;
  if (!dst) return fail(RLXPP_ERR_INVALID, "null destination");
  cudaStream_t st = as_stream(cuda_stream);
  const size_t bytes = sizeof(rlxpp_state) * g->n;
  if (on_device(dst)) {
    cudaError_t e = launch_export(g->view(), g->level_p, dst, st);
    if (e != cudaSuccess) return fail(cuda_status(e), std::string("export: ") + cudaGetErrorString(e));
    return RLXPP_OK;
  }
  void* dev = nullptr;
  RLX_CUDA(dev_malloc_async(&dev, bytes, st));
  cudaError_t e = launch_export(g->view(), g->level_p, static_cast<rlxpp_state*>(dev), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dev, st);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("export: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

rlxpp_status rlxpp_set_state(rlxpp_gen* g, const rlxpp_state* src, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  if (g->n == 0) return RLXPP_OK;
  if (!src) return fail(RLXPP_ERR_INVALID, "null source");
  cudaStream_t st = as_stream(cuda_stream);
  Staged ss;
  if (rlxpp_status s = stage_in(src, sizeof(rlxpp_state) * g->n, st, ss)) return s;
  cudaError_t e = launch_import(g->view(), g->level_p, g->n_levels,
                                static_cast<const rlxpp_state*>(ss.dev), st);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("import: ") + cudaGetErrorString(e));
  g->level_host_stale = true;  // levels may have changed; the next request plan re-reads them
  return RLXPP_OK;
}

rlxpp_status rlxpp_sync(rlxpp_gen* g, void* cuda_stream) {
  if (rlxpp_status s = check_gen(g)) return s;
  cudaStream_t st = as_stream(cuda_stream);
  int h = 0;
  RLX_CUDA(cudaMemcpyAsync(&h, g->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  RLX_CUDA(cudaMemsetAsync(g->status, 0, sizeof(int), st));
  RLX_CUDA(cudaStreamSynchronize(st));
  if (h == RLXPP_ERR_INVALID) return fail(RLXPP_ERR_INVALID, "a kernel rejected its input");
  if (h == RLXPP_ERR_TIMEOUT) return fail(RLXPP_ERR_TIMEOUT, "a bounded device wait gave up");
  if (h != 0) return fail(RLXPP_ERR_CUDA, "unknown device status");
  return RLXPP_OK;
}

rlxpp_status rlxpp_set_path(rlxpp_gen* g, uint32_t path) {
  if (rlxpp_status s = check_gen(g)) return s;
  if (path != RLXPP_PATH_IMAD && path != RLXPP_PATH_TENSOR && path != RLXPP_PATH_WARP)
    return fail(RLXPP_ERR_INVALID, "unknown path");
  if (path == RLXPP_PATH_TENSOR && !g->tc_matrix) return fail(RLXPP_ERR_CUDA, "tensor matrix missing");
  RLX_CUDA(cudaDeviceSynchronize());  // no draw of the old path may still run
  g->path = path;
  return RLXPP_OK;
}

uint32_t rlxpp_get_path(const rlxpp_gen* g) { return g ? g->path : 0u; }

uint64_t rlxpp_num_streams(const rlxpp_gen* g) { return g ? g->n : 0; }

const char* rlxpp_last_error(void) { return g_last_error.c_str(); }

void rlxpp_destroy(rlxpp_gen* g) {
  RLX_LOG_CALL("destroy gen %p", (void*)g);
  free_gen(g);
}

rlxpp_status rlxpp_test_fail_alloc(int64_t after) {
  g_fail_alloc.store(after < 0 ? -1 : after);
  return RLXPP_OK;
}

// ---- unit-test entry points --------------------------------------------------------
static rlxpp_status run_test(int op, const void* x, const void* y, void* out, void* carry,
                             uint64_t n, void* cuda_stream) {
  if (n == 0) return RLXPP_OK;
  if (!x || !out) return fail(RLXPP_ERR_INVALID, "null test buffer");
  cudaError_t e = launch_test(op, static_cast<const uint64_t*>(x), static_cast<const uint64_t*>(y),
                              static_cast<uint64_t*>(out), static_cast<uint32_t*>(carry), n,
                              as_stream(cuda_stream));
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("test kernel: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}

rlxpp_status rlxpp_test_multiply9x9(const uint64_t* x, const uint64_t* y, uint64_t* out, uint64_t n,
                                    void* cuda_stream) {
  if (n && !y) return fail(RLXPP_ERR_INVALID, "null y");
  return run_test(kTestMultiply, x, y, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_mod_m(const uint64_t* in, uint64_t* out, uint64_t n, void* cuda_stream) {
  return run_test(kTestModM, in, nullptr, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_mul_mod(const uint64_t* x, const uint64_t* y, uint64_t* out, uint64_t n,
                                void* cuda_stream) {
  if (n && !y) return fail(RLXPP_ERR_INVALID, "null y");
  return run_test(kTestMulMod, x, y, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_to_ranlux(const uint64_t* x, uint64_t* d, uint32_t* carry, uint64_t n,
                                  void* cuda_stream) {
  if (n && !carry) return fail(RLXPP_ERR_INVALID, "null carry");
  return run_test(kTestToRanlux, x, nullptr, d, carry, n, cuda_stream);
}
rlxpp_status rlxpp_test_to_lcg(const uint64_t* d, const uint32_t* carry, uint64_t* x, uint64_t n,
                               void* cuda_stream) {
  if (n && !carry) return fail(RLXPP_ERR_INVALID, "null carry");
  return run_test(kTestToLcg, d, nullptr, x, const_cast<uint32_t*>(carry), n, cuda_stream);
}
rlxpp_status rlxpp_test_f64_from48(const uint64_t* v, uint64_t* out, uint64_t n, void* cuda_stream) {
  return run_test(kTestF64, v, nullptr, out, nullptr, n, cuda_stream);
}
static rlxpp_status warp_test(int op, const uint64_t* in, uint64_t* out, uint32_t* carry, uint64_t n,
                              void* cuda_stream) {
  if (n == 0) return RLXPP_OK;
  if (!in || !out || (op == 1 && !carry)) return fail(RLXPP_ERR_INVALID, "null test buffer");
  cudaError_t e = launch_warp_test(op, in, out, carry, n, as_stream(cuda_stream));
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("warp test kernel: ") + cudaGetErrorString(e));
  return RLXPP_OK;
}
rlxpp_status rlxpp_test_warp_mod_m(const uint64_t* in, uint64_t* out, uint64_t n, void* cuda_stream) {
  return warp_test(0, in, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_warp_to_ranlux(const uint64_t* x, uint64_t* d, uint32_t* carry, uint64_t n,
                                       void* cuda_stream) {
  return warp_test(1, x, d, carry, n, cuda_stream);
}
rlxpp_status rlxpp_test_neg_ln48(const uint64_t* w, uint64_t* out, uint64_t n, void* cuda_stream) {
  return run_test(kTestNegLn48, w, nullptr, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_cos_sin_2pi48(const uint64_t* v, uint64_t* out, uint64_t n, void* cuda_stream) {
  return run_test(kTestCosSin2Pi48, v, nullptr, out, nullptr, n, cuda_stream);
}
rlxpp_status rlxpp_test_box_muller48(const uint64_t* v, uint64_t* out, uint64_t n, void* cuda_stream) {
  return run_test(kTestBoxMuller48, v, nullptr, out, nullptr, n, cuda_stream);
}

static rlxpp_status tc_test(uint32_t p, const uint64_t* x, uint64_t* out, uint64_t n, void* cuda_stream,
                            bool issue);

rlxpp_status rlxpp_test_tc_mulmod(uint32_t p, const uint64_t* x, uint64_t* out, uint64_t n, void* cuda_stream) {
  return tc_test(p, x, out, n, cuda_stream, true);
}

rlxpp_status rlxpp_test_tc_timeout(uint64_t* scratch, void* cuda_stream) {
  if (!scratch) return fail(RLXPP_ERR_INVALID, "null scratch");
  return tc_test(1, scratch, scratch, 1, cuda_stream, false);
}

static rlxpp_status tc_test(uint32_t p, const uint64_t* x, uint64_t* out, uint64_t n, void* cuda_stream,
                            bool issue) {
  if (p == 0) return fail(RLXPP_ERR_INVALID, "need p >= 1");
  if (n == 0) return RLXPP_OK;
  if (!x || !out) return fail(RLXPP_ERR_INVALID, "null test buffer");
  cudaStream_t st = as_stream(cuda_stream);
  uint32_t *lux = nullptr, *table = nullptr;
  void* mat = nullptr;
  int* status = nullptr;
  cudaError_t e = dev_malloc(&lux, sizeof(uint32_t) * 18);
  if (e == cudaSuccess) e = dev_malloc(&table, sizeof(uint32_t) * kTableLimbs);
  if (e == cudaSuccess) e = dev_malloc(&mat, tc_matrix_bytes());
  if (e == cudaSuccess) e = dev_malloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = launch_level_setup(p, lux, table, st);
  if (e == cudaSuccess) e = launch_tc_matrix(lux, mat, st);
  if (e == cudaSuccess) e = launch_tc_mulmod(mat, x, out, n, status, st, issue);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(lux);
  cudaFree(table);
  cudaFree(mat);
  cudaFree(status);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("tensor test: ") + cudaGetErrorString(e));
  if (h) return fail((rlxpp_status)h, "tensor test: a bounded device wait gave up");
  return RLXPP_OK;
}

rlxpp_status rlxpp_luxury_multiplier(uint32_t p, uint64_t* out9) {
  if (p == 0 || !out9) return fail(RLXPP_ERR_INVALID, "need p >= 1 and an output");
  uint32_t *lux = nullptr, *table = nullptr;
  RLX_CUDA(dev_malloc(&lux, sizeof(uint32_t) * 18));
  cudaError_t e = dev_malloc(&table, sizeof(uint32_t) * kTableLimbs);
  if (e == cudaSuccess) e = launch_level_setup(p, lux, table, nullptr);
  uint32_t h[18] = {};
  if (e == cudaSuccess) e = cudaMemcpy(h, lux, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(lux);
  cudaFree(table);
  if (e != cudaSuccess) return fail(cuda_status(e), std::string("luxury multiplier: ") + cudaGetErrorString(e));
  for (int k = 0; k < 9; ++k) out9[k] = ((uint64_t)h[2 * k + 1] << 32) | h[2 * k];
  return RLXPP_OK;
}

}  // extern "C"
