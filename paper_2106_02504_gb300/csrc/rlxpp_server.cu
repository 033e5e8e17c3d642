// Continuous-batching request loop over resident streams, on the host in C++ (the
// device work of each batch is rlxpp_draw_requests).  Every resident stream keeps its
// state on the device; a request asks for `count` u24 integers or doubles from one
// stream and gets the next segment of that stream at submission (its start block and
// read position follow from a host-side cursor: 24 numbers per block, 2 per double, a
// lone leftover number skipped), so it runs by jump-ahead before, after or beside any
// other request.  A request is admitted when its output fits a device arena (first fit,
// 256-byte granules, coalescing), launched with what else is admitted as one batch on
// one of several CUDA streams while earlier batches run, copied to a page-locked mirror
// of the arena (the batch's small requests first, one copy per run of adjacent blocks,
// then each large one by itself, smallest first, each group behind its own event) and
// completed when its group's event has fired.  Admission can be bounded by the bytes
// waiting for the arena (rejected requests take no numbers from their stream); a request
// not yet launched can be cancelled (its segment is skipped).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rlxpp_internal.h"

using namespace rlxpp;

namespace {

constexpr uint64_t kBlockWords = 24;  // RANLUX numbers per block
constexpr uint64_t kGranule = 256;    // arena allocation unit

enum ReqState { kWaiting = 0, kAdmitted = 1, kLaunched = 2, kDone = 3 };

struct Req {
  rlxpp_served rec{};                     // public record (rid, stream, segment, times)
  uint64_t reserved = 0;                  // arena bytes held
  int state = kWaiting;
};

// First-fit allocator over [0, size) with a sorted, coalesced free list.
class Arena {
 public:
  explicit Arena(uint64_t size) : size_(size) { free_.push_back({0, size}); }
  bool alloc(uint64_t nbytes, uint64_t& off, uint64_t& len) {
    const uint64_t n = (nbytes + kGranule - 1) / kGranule * kGranule;
    for (size_t k = 0; k < free_.size(); ++k) {
      if (free_[k].second >= n) {
        off = free_[k].first;
        len = n;
        if (free_[k].second == n)
          free_.erase(free_.begin() + (long)k);
        else
          free_[k] = {off + n, free_[k].second - n};
        used_ += n;
        return true;
      }
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    used_ -= n;
    auto it = std::lower_bound(free_.begin(), free_.end(), std::make_pair(off, (uint64_t)0));
    it = free_.insert(it, {off, n});
    size_t k = (size_t)(it - free_.begin());
    if (k + 1 < free_.size() && free_[k].first + free_[k].second == free_[k + 1].first) {
      free_[k].second += free_[k + 1].second;
      free_.erase(free_.begin() + (long)k + 1);
    }
    if (k > 0 && free_[k - 1].first + free_[k - 1].second == free_[k].first) {
      free_[k - 1].second += free_[k].second;
      free_.erase(free_.begin() + (long)k);
    }
  }
  uint64_t size() const { return size_; }
  uint64_t used() const { return used_; }

 private:
  uint64_t size_, used_ = 0;
  std::vector<std::pair<uint64_t, uint64_t>> free_;  // (offset, length), sorted
};

struct Group {
  cudaEvent_t ev;
  std::vector<Req*> reqs;
};
struct InFlight {
  int si;
  std::deque<Group> groups;
  cudaEvent_t t[3];  // timing events: batch start, request kernel end, copies end
};

double now_s() {
  using clk = std::chrono::steady_clock;
  static const clk::time_point origin = clk::now();
  return std::chrono::duration<double>(clk::now() - origin).count();
}

}  // namespace

struct rlxpp_server {
  rlxpp_gen* gen = nullptr;
  uint64_t n_streams = 0;
  unsigned char* dev = nullptr;
  unsigned char* host = nullptr;  // page-locked mirror (null: results stay on the device)
  std::unique_ptr<Arena> arena;
  std::vector<cudaStream_t> streams;
  std::deque<int> free_streams;
  std::deque<Req*> waiting, admitted;
  std::deque<InFlight> inflight;
  std::vector<uint64_t> cur_block;
  std::vector<uint8_t> cur_pos;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> live;  // rid -> not yet taken
  std::deque<uint64_t> done_order;                          // completed, in completion order
  std::unordered_map<uint64_t, std::vector<unsigned char>> results;
  std::vector<cudaEvent_t> event_pool;
  std::vector<rlxpp_request> batch;  // scratch
  uint32_t max_batch = 512;
  uint64_t small_bytes = 1 << 20, max_queued = 0, queued = 0;
  bool keep_results = false;
  double t0 = 0;  // time origin of arrival times
  uint64_t n_done = 0, n_rejected = 0, n_cancelled = 0;
  double max_launch_s = 0;   // longest host time of one batch launch (rlxpp_draw_requests)
  uint64_t slow_launches = 0;  // launches of 1 ms or more
  std::vector<cudaEvent_t> timing_pool;  // events with timing, three per batch
  uint64_t batches_timed = 0;
  double kernel_s_sum = 0, kernel_s_max = 0, copy_s_sum = 0, copy_s_max = 0;
};

namespace {

rlxpp_status cuda_fail(cudaError_t e, const char* what) {
  return set_last_error(e == cudaErrorMemoryAllocation ? RLXPP_ERR_NOMEM : RLXPP_ERR_CUDA,
                        (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

// Stream position after `count` values of `kind` read from (block, pos).
void advance_cursor(uint64_t& block, uint8_t& pos, uint32_t kind, int64_t count) {
  const uint32_t need = kind == RLXPP_KIND_F64 ? 2 : 1;
  const uint64_t per = kBlockWords / need;
  const uint64_t room = pos + need <= kBlockWords ? (kBlockWords - pos) / need : 0;
  const uint64_t head = std::min<uint64_t>((uint64_t)count, room);
  const uint64_t rest = (uint64_t)count - head;
  if (rest == 0) {
    pos = (uint8_t)(pos + head * need);
    return;
  }
  const uint64_t refills = (rest + per - 1) / per;
  const uint64_t last = rest - (refills - 1) * per;
  block += refills;
  pos = (uint8_t)(last * need);
}

rlxpp_status get_event(rlxpp_server* s, cudaEvent_t& ev) {
  if (!s->event_pool.empty()) {
    ev = s->event_pool.back();
    s->event_pool.pop_back();
    return RLXPP_OK;
  }
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  return e == cudaSuccess ? RLXPP_OK : cuda_fail(e, "server event");
}

rlxpp_status get_timing_event(rlxpp_server* s, cudaEvent_t& ev) {
  if (!s->timing_pool.empty()) {
    ev = s->timing_pool.back();
    s->timing_pool.pop_back();
    return RLXPP_OK;
  }
  cudaError_t e = cudaEventCreate(&ev);
  return e == cudaSuccess ? RLXPP_OK : cuda_fail(e, "server timing event");
}

// Device times of a completed batch (its last copy is done, so all three events have
// completed); the events go back to the pool.
void record_batch_times(rlxpp_server* s, InFlight& f) {
  float k_ms = 0, c_ms = 0;
  if (cudaEventElapsedTime(&k_ms, f.t[0], f.t[1]) == cudaSuccess &&
      cudaEventElapsedTime(&c_ms, f.t[1], f.t[2]) == cudaSuccess) {
    ++s->batches_timed;
    s->kernel_s_sum += k_ms * 1e-3;
    s->kernel_s_max = std::max(s->kernel_s_max, k_ms * 1e-3);
    s->copy_s_sum += c_ms * 1e-3;
    s->copy_s_max = std::max(s->copy_s_max, c_ms * 1e-3);
  } else {
    cudaGetLastError();
  }
  for (cudaEvent_t& ev : f.t) s->timing_pool.push_back(ev);
}

void admit(rlxpp_server* s) {
  while (!s->waiting.empty()) {
    Req* r = s->waiting.front();
    uint64_t off, len;
    if (!s->arena->alloc(std::max<uint64_t>(r->rec.nbytes, 1), off, len)) return;
    r->rec.offset = off;
    r->reserved = len;
    r->state = kAdmitted;
    s->waiting.pop_front();
    s->queued -= r->rec.nbytes;
    s->admitted.push_back(r);
  }
}

rlxpp_status dispatch(rlxpp_server* s) {
  while (!s->admitted.empty() && !s->free_streams.empty()) {
    const size_t nb = std::min<size_t>(s->max_batch, s->admitted.size());
    std::vector<Req*> reqs(s->admitted.begin(), s->admitted.begin() + (long)nb);
    s->admitted.erase(s->admitted.begin(), s->admitted.begin() + (long)nb);
    const int si = s->free_streams.front();
    s->free_streams.pop_front();
    cudaStream_t st = s->streams[si];
    s->batch.resize(nb);
    for (size_t k = 0; k < nb; ++k) {
      const rlxpp_served& q = reqs[k]->rec;
      s->batch[k] = rlxpp_request{q.stream, q.skip, q.pos, q.kind, q.count,
                                  q.offset / (q.kind == RLXPP_KIND_F64 ? 8 : 4)};
    }
    InFlight f{si, {}, {}};
    for (cudaEvent_t& ev : f.t)
      if (rlxpp_status es = get_timing_event(s, ev)) return es;
    cudaError_t et = cudaEventRecord(f.t[0], st);
    if (et != cudaSuccess) return cuda_fail(et, "server event record");
    const double l0 = now_s();
    if (rlxpp_status rs = rlxpp_draw_requests(s->gen, s->batch.data(), nb, reinterpret_cast<uint32_t*>(s->dev),
                                              reinterpret_cast<double*>(s->dev), 0, st))
      return rs;
    const double dl = now_s() - l0;
    s->max_launch_s = std::max(s->max_launch_s, dl);
    if (dl >= 1e-3) ++s->slow_launches;
    et = cudaEventRecord(f.t[1], st);
    if (et != cudaSuccess) return cuda_fail(et, "server event record");
    auto close_group = [&](std::vector<Req*>&& members) -> rlxpp_status {
      cudaEvent_t ev;
      if (rlxpp_status es = get_event(s, ev)) return es;
      cudaError_t e = cudaEventRecord(ev, st);
      if (e != cudaSuccess) return cuda_fail(e, "server event record");
      f.groups.push_back(Group{ev, std::move(members)});
      return RLXPP_OK;
    };
    if (s->host) {
      // small requests first, one copy per run of adjacent arena blocks
      std::vector<Req*> small, large;
      for (Req* r : reqs) (r->rec.nbytes < s->small_bytes ? small : large).push_back(r);
      std::sort(large.begin(), large.end(), [](const Req* a, const Req* b) { return a->rec.nbytes < b->rec.nbytes; });
      if (!small.empty()) {
        std::vector<std::pair<uint64_t, uint64_t>> spans;
        for (Req* r : small)
          if (r->rec.nbytes) spans.push_back({r->rec.offset, r->reserved});
        std::sort(spans.begin(), spans.end());
        for (size_t k = 0; k < spans.size();) {
          uint64_t a = spans[k].first, ln = spans[k].second;
          while (k + 1 < spans.size() && spans[k + 1].first == a + ln) ln += spans[++k].second;
          cudaError_t e = cudaMemcpyAsync(s->host + a, s->dev + a, ln, cudaMemcpyDeviceToHost, st);
          if (e != cudaSuccess) return cuda_fail(e, "server copy");
          ++k;
        }
        if (rlxpp_status gs = close_group(std::move(small))) return gs;
      }
      for (Req* r : large) {
        cudaError_t e = cudaMemcpyAsync(s->host + r->rec.offset, s->dev + r->rec.offset, r->rec.nbytes,
                                        cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "server copy");
        if (rlxpp_status gs = close_group(std::vector<Req*>{r})) return gs;
      }
    } else {
      if (rlxpp_status gs = close_group(std::move(reqs))) return gs;
    }
    et = cudaEventRecord(f.t[2], st);  // after every copy of the batch
    if (et != cudaSuccess) return cuda_fail(et, "server event record");
    const double t = now_s() - s->t0;
    for (const Group& g : f.groups)
      for (Req* r : g.reqs) {
        r->rec.launch = t;
        r->state = kLaunched;
      }
    s->inflight.push_back(std::move(f));
  }
  return RLXPP_OK;
}

// Retire every request whose group's event has fired (a stream's groups finish in
// order); a CUDA stream is free again once its batch's last group is done.  With
// wait_first, first wait for the oldest batch's next group.
rlxpp_status complete(rlxpp_server* s, bool wait_first) {
  if (wait_first && !s->inflight.empty()) {
    cudaError_t e = cudaEventSynchronize(s->inflight.front().groups.front().ev);
    if (e != cudaSuccess) return cuda_fail(e, "server wait");
  }
  std::deque<InFlight> keep;
  while (!s->inflight.empty()) {
    InFlight f = std::move(s->inflight.front());
    s->inflight.pop_front();
    while (!f.groups.empty()) {
      cudaError_t e = cudaEventQuery(f.groups.front().ev);
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) return cuda_fail(e, "server event query");
      Group g = std::move(f.groups.front());
      f.groups.pop_front();
      const double t = now_s() - s->t0;
      for (Req* r : g.reqs) {
        r->rec.done = t;
        r->state = kDone;
        if (s->keep_results && s->host && r->rec.nbytes)
          s->results[r->rec.rid].assign(s->host + r->rec.offset, s->host + r->rec.offset + r->rec.nbytes);
        s->arena->release(r->rec.offset, r->reserved);
        s->done_order.push_back(r->rec.rid);
        ++s->n_done;
      }
      s->event_pool.push_back(g.ev);
    }
    if (f.groups.empty()) {
      // the batch's last group is done; its timing events follow within the stream
      if (cudaEventSynchronize(f.t[2]) == cudaSuccess) record_batch_times(s, f);
      else for (cudaEvent_t& ev : f.t) s->timing_pool.push_back(ev);
      s->free_streams.push_back(f.si);
    } else
      keep.push_back(std::move(f));
  }
  s->inflight = std::move(keep);
  return RLXPP_OK;
}

rlxpp_status pump(rlxpp_server* s) {
  if (rlxpp_status st = complete(s, false)) return st;
  admit(s);
  return dispatch(s);
}

bool busy(const rlxpp_server* s) { return !s->waiting.empty() || !s->admitted.empty() || !s->inflight.empty(); }

void free_server(rlxpp_server* s) {
  if (!s) return;
  for (auto st : s->streams)
    if (st) cudaStreamSynchronize(st);
  for (auto& f : s->inflight)
    for (auto& g : f.groups) cudaEventDestroy(g.ev);
  for (auto ev : s->event_pool) cudaEventDestroy(ev);
  for (auto& f : s->inflight)
    for (auto ev : f.t) cudaEventDestroy(ev);
  for (auto ev : s->timing_pool) cudaEventDestroy(ev);
  for (auto st : s->streams)
    if (st) cudaStreamDestroy(st);
  cudaFree(s->dev);
  cudaFreeHost(s->host);
  delete s;
}

}  // namespace

extern "C" {

rlxpp_status rlxpp_server_create(rlxpp_gen* gen, uint64_t pool_bytes, uint32_t n_cuda_streams, uint32_t max_batch,
                                 uint64_t small_bytes, uint64_t max_queued_bytes, uint32_t flags,
                                 rlxpp_server** out) {
  if (!out) return set_last_error(RLXPP_ERR_INVALID, "null server output");
  *out = nullptr;
  if (!gen) return set_last_error(RLXPP_ERR_INVALID, "null generator handle");
  if (pool_bytes < kGranule || n_cuda_streams == 0 || n_cuda_streams > 64 || max_batch == 0)
    return set_last_error(RLXPP_ERR_INVALID, "need pool_bytes >= 256, 1..64 CUDA streams, max_batch >= 1");
  if (flags & ~(RLXPP_SERVER_COPY_TO_HOST | RLXPP_SERVER_KEEP_RESULTS))
    return set_last_error(RLXPP_ERR_INVALID, "unknown server flags");
  const uint64_t n = rlxpp_num_streams(gen);
  auto* s = new rlxpp_server();
  s->gen = gen;
  s->n_streams = n;
  s->arena.reset(new Arena(pool_bytes / kGranule * kGranule));  // whole granules
  s->max_batch = max_batch;
  s->small_bytes = small_bytes;
  s->max_queued = max_queued_bytes;
  s->keep_results = (flags & RLXPP_SERVER_KEEP_RESULTS) != 0;
  s->cur_block.assign(n, 0);
  s->cur_pos.assign(n, 0);
  cudaError_t e = cudaMalloc(&s->dev, pool_bytes);
  if (e == cudaSuccess && (flags & RLXPP_SERVER_COPY_TO_HOST))
    e = cudaHostAlloc(reinterpret_cast<void**>(&s->host), pool_bytes, cudaHostAllocDefault);
  s->streams.assign(n_cuda_streams, nullptr);
  for (uint32_t k = 0; e == cudaSuccess && k < n_cuda_streams; ++k) {
    e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
    s->free_streams.push_back((int)k);
  }
  if (e != cudaSuccess) {
    rlxpp_status st = cuda_fail(e, "server create");
    free_server(s);
    return st;
  }
  s->t0 = now_s();
  *out = s;
  return RLXPP_OK;
}

void rlxpp_server_destroy(rlxpp_server* s) { free_server(s); }

rlxpp_status rlxpp_server_submit(rlxpp_server* s, uint64_t rid, uint64_t stream, uint32_t kind, int64_t count,
                                 double arrival, int* accepted) {
  if (!s || !accepted) return set_last_error(RLXPP_ERR_INVALID, "null server or output");
  *accepted = 0;
  if (stream >= s->n_streams || count < 0 || (kind != RLXPP_KIND_U24 && kind != RLXPP_KIND_F64))
    return set_last_error(RLXPP_ERR_INVALID, "bad request");
  if (s->live.count(rid)) return set_last_error(RLXPP_ERR_INVALID, "request id in use");
  const uint64_t nbytes = (uint64_t)count * (kind == RLXPP_KIND_F64 ? 8 : 4);
  const uint64_t held = (std::max<uint64_t>(nbytes, 1) + kGranule - 1) / kGranule * kGranule;
  if (held > s->arena->size() || (s->max_queued && s->queued + nbytes > s->max_queued)) {
    ++s->n_rejected;  // takes no numbers from the stream
    return RLXPP_OK;
  }
  auto r = std::make_unique<Req>();
  r->rec.rid = rid;
  r->rec.stream = stream;
  r->rec.kind = kind;
  r->rec.count = count;
  r->rec.nbytes = nbytes;
  r->rec.skip = s->cur_block[stream];
  r->rec.pos = s->cur_pos[stream];
  r->rec.arrival = arrival < 0 ? now_s() - s->t0 : arrival;
  advance_cursor(s->cur_block[stream], s->cur_pos[stream], kind, count);
  s->queued += nbytes;
  s->waiting.push_back(r.get());
  s->live[rid] = std::move(r);
  *accepted = 1;
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_cancel(rlxpp_server* s, uint64_t rid, int* cancelled) {
  if (!s || !cancelled) return set_last_error(RLXPP_ERR_INVALID, "null server or output");
  *cancelled = 0;
  auto it = s->live.find(rid);
  if (it == s->live.end() || it->second->state > kAdmitted) return RLXPP_OK;
  Req* r = it->second.get();
  if (r->state == kWaiting) {
    s->waiting.erase(std::find(s->waiting.begin(), s->waiting.end(), r));
    s->queued -= r->rec.nbytes;
  } else {
    s->admitted.erase(std::find(s->admitted.begin(), s->admitted.end(), r));
    s->arena->release(r->rec.offset, r->reserved);
  }
  s->live.erase(it);
  ++s->n_cancelled;
  *cancelled = 1;
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_pump(rlxpp_server* s, int wait_for_one) {
  if (!s) return set_last_error(RLXPP_ERR_INVALID, "null server");
  if (wait_for_one && !s->inflight.empty())
    if (rlxpp_status st = complete(s, true)) return st;
  return pump(s);
}

rlxpp_status rlxpp_server_drain(rlxpp_server* s) {
  if (!s) return set_last_error(RLXPP_ERR_INVALID, "null server");
  while (busy(s)) {
    if (rlxpp_status st = pump(s)) return st;
    if (!s->inflight.empty() && (s->free_streams.empty() || s->admitted.empty()))
      if (rlxpp_status st = complete(s, true)) return st;
  }
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_stats(const rlxpp_server* s, rlxpp_server_state* out) {
  if (!s || !out) return set_last_error(RLXPP_ERR_INVALID, "null server or output");
  out->waiting = s->waiting.size();
  out->admitted = s->admitted.size();
  uint64_t groups = 0;
  for (const auto& f : s->inflight) groups += f.groups.size();
  out->inflight_groups = groups;
  out->arena_used = s->arena->used();
  out->queued_bytes = s->queued;
  out->done = s->n_done;
  out->rejected = s->n_rejected;
  out->cancelled = s->n_cancelled;
  out->max_launch_us = (uint64_t)(s->max_launch_s * 1e6);
  out->slow_launches = s->slow_launches;
  out->batches_timed = s->batches_timed;
  out->kernel_us_sum = (uint64_t)(s->kernel_s_sum * 1e6);
  out->kernel_us_max = (uint64_t)(s->kernel_s_max * 1e6);
  out->copy_us_sum = (uint64_t)(s->copy_s_sum * 1e6);
  out->copy_us_max = (uint64_t)(s->copy_s_max * 1e6);
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_take_done(rlxpp_server* s, rlxpp_served* out, uint64_t max, uint64_t* n) {
  if (!s || !n || (max && !out)) return set_last_error(RLXPP_ERR_INVALID, "null server or output");
  *n = 0;
  while (*n < max && !s->done_order.empty()) {
    const uint64_t rid = s->done_order.front();
    s->done_order.pop_front();
    auto it = s->live.find(rid);
    out[(*n)++] = it->second->rec;
    s->live.erase(it);
  }
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_result(rlxpp_server* s, uint64_t rid, void* dst, uint64_t nbytes) {
  if (!s || (nbytes && !dst)) return set_last_error(RLXPP_ERR_INVALID, "null server or output");
  auto it = s->results.find(rid);
  if (it == s->results.end()) {
    if (nbytes == 0) return RLXPP_OK;
    return set_last_error(RLXPP_ERR_INVALID, "no kept result for this request");
  }
  if (it->second.size() != nbytes) return set_last_error(RLXPP_ERR_INVALID, "result size differs");
  std::memcpy(dst, it->second.data(), nbytes);
  s->results.erase(it);
  return RLXPP_OK;
}

rlxpp_status rlxpp_server_run_trace(rlxpp_server* s, uint64_t n, const double* arrival, const uint64_t* stream,
                                    const int64_t* count, const uint8_t* is_f64, double* latency) {
  if (!s || (n && (!arrival || !stream || !count || !is_f64 || !latency)))
    return set_last_error(RLXPP_ERR_INVALID, "null server or trace array");
  if (busy(s) || !s->live.empty())
    return set_last_error(RLXPP_ERR_INVALID, "a trace needs an idle server with every result taken");
  for (uint64_t k = 0; k < n; ++k) latency[k] = -1.0;  // rejected requests stay at -1
  // the launch and device times that rlxpp_server_stats reports cover this trace only
  s->max_launch_s = 0.0;
  s->slow_launches = 0;
  s->batches_timed = 0;
  s->kernel_s_sum = s->kernel_s_max = 0.0;
  s->copy_s_sum = s->copy_s_max = 0.0;
  s->t0 = now_s();
  uint64_t i = 0;
  const uint64_t base_rid = 0;  // request i of the trace has id i
  while (i < n || busy(s)) {
    const double t = now_s() - s->t0;
    while (i < n && arrival[i] <= t) {
      int ok = 0;
      if (rlxpp_status st = rlxpp_server_submit(s, base_rid + i, stream[i],
                                                is_f64[i] ? RLXPP_KIND_F64 : RLXPP_KIND_U24, count[i],
                                                arrival[i], &ok))
        return st;
      ++i;
    }
    if (rlxpp_status st = pump(s)) return st;
    while (!s->done_order.empty()) {  // latencies of the finished ones
      const uint64_t rid = s->done_order.front();
      s->done_order.pop_front();
      auto it = s->live.find(rid);
      latency[rid - base_rid] = it->second->rec.done - it->second->rec.arrival;
      s->live.erase(it);
    }
    if (i < n && s->waiting.empty() && s->admitted.empty()) {
      const double gap = arrival[i] - (now_s() - s->t0);
      if (gap > 2e-4 && s->inflight.empty())
        std::this_thread::sleep_for(std::chrono::duration<double>(std::min(gap, 1e-3)));
    }
  }
  return RLXPP_OK;
}

}  // extern "C"
