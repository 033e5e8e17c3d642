"""Continuous-batching request loop over resident RANLUX++ streams.

Every resident stream keeps its state on the device (created once, never rewritten by
the loop).  A request asks for `count` u24 integers or doubles from one stream; at
arrival it is given the next segment of that stream — its start block and read
position follow from the stream's host-side cursor by position arithmetic (24 numbers
per block, 2 per double, a lone leftover number skipped) — so it can run before,
after or beside any other request: the device starts it by jump-ahead
(rlxpp_draw_requests with skip = start block).  A request is admitted when its output
fits in a fixed device-memory arena, launched with whatever else is admitted as one
batch on one of several CUDA streams while earlier batches still run, copied to a
pinned host mirror of the arena, and completed when its copy has finished: the small
requests of a batch are copied first (adjacent blocks in one copy), then each large one
by itself, smallest first, each group with its own event.

Admission: with a bound on the bytes waiting for the arena (max_queued_bytes), a request
that would exceed it, or one larger than the whole arena, is rejected at submission and
takes no numbers from its stream (the next request of that stream gets the segment).
Cancellation: a request not yet launched can be cancelled; its segment of the stream is
then skipped, as if drawn and discarded.
"""
from __future__ import annotations

import collections
import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import _rlxpp as B

KIND_U24, KIND_F64 = B.RLXPP_KIND_U24, B.RLXPP_KIND_F64
_ALIGN = 256


def advance_cursor(block, pos, kind, count):
    """Stream position after `count` values of `kind` starting at (block, pos)."""
    need = 2 if kind == KIND_F64 else 1
    per = 24 // need
    room = (24 - pos) // need if pos + need <= 24 else 0
    head = min(count, room)
    rest = count - head
    if rest == 0:
        return block, pos + head * need
    refills = -(-rest // per)
    last = rest - (refills - 1) * per
    return block + refills, last * need


class Arena:
    """First-fit allocator over [0, size) bytes with coalescing free list."""

    def __init__(self, size):
        self.size = size
        self.free = [(0, size)]     # sorted (offset, length)
        self.used = 0

    def alloc(self, nbytes):
        n = -(-nbytes // _ALIGN) * _ALIGN
        for k, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, ln - n)
                self.used += n
                return off, n
        return None

    def release(self, off, n):
        self.used -= n
        lo, hi = 0, len(self.free)
        while lo < hi:
            mid = (lo + hi) // 2
            if self.free[mid][0] < off:
                lo = mid + 1
            else:
                hi = mid
        self.free.insert(lo, (off, n))
        if lo + 1 < len(self.free) and self.free[lo][0] + self.free[lo][1] == self.free[lo + 1][0]:
            self.free[lo] = (off, self.free[lo][1] + self.free[lo + 1][1])
            self.free.pop(lo + 1)
        if lo > 0 and self.free[lo - 1][0] + self.free[lo - 1][1] == self.free[lo][0]:
            self.free[lo - 1] = (self.free[lo - 1][0], self.free[lo - 1][1] + self.free[lo][1])
            self.free.pop(lo)


@dataclass
class Request:
    rid: int
    stream: int
    kind: int
    count: int
    arrival: float
    skip: int = 0
    pos: int = 0
    offset: int = -1          # byte offset in the arena
    nbytes: int = 0
    reserved: int = 0
    launch: float = 0.0
    done: float = 0.0
    status: str = "waiting"   # waiting, admitted, launched, done, rejected, cancelled
    result: np.ndarray | None = field(default=None, repr=False)


class Server:
    def __init__(self, n_resident, luxury=2048, seeds=None, pool_bytes=1 << 30, n_cuda_streams=4,
                 max_batch=512, keep_results=False, copy_to_host=True, small_bytes=1 << 20,
                 max_queued_bytes=None):
        import torch
        self.torch = torch
        if seeds is None:
            seeds = np.arange(1, n_resident + 1, dtype=np.uint64)
        self.gen = B.Generator(n_resident, [luxury], torch.from_numpy(np.asarray(seeds, np.uint64).view(np.int64)).cuda())
        self.n = n_resident
        self.cur_block = [0] * n_resident
        self.cur_pos = [0] * n_resident
        self.dev = torch.empty(pool_bytes, dtype=torch.uint8, device="cuda")
        self.host = torch.empty(pool_bytes, dtype=torch.uint8).pin_memory() if copy_to_host else None
        self.arena = Arena(pool_bytes // _ALIGN * _ALIGN)  # whole granules
        self.streams = [torch.cuda.Stream() for _ in range(n_cuda_streams)]
        self.free_streams = collections.deque(range(n_cuda_streams))
        self.waiting = collections.deque()     # arrived, not admitted (FIFO)
        self.admitted = collections.deque()    # admitted, not launched
        self.inflight = collections.deque()    # (stream index, deque of (event, [requests]))
        self.max_batch = max_batch
        self.small_bytes = small_bytes   # requests below this size share one copy group
        self.keep_results = keep_results
        self.finished = []
        self.max_queued_bytes = max_queued_bytes
        self.queued_bytes = 0      # bytes of the requests waiting for the arena
        self.pending = {}          # rid -> request not yet launched
        self.rejected = []
        self.cancelled = []
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    # -- request life cycle -----------------------------------------------------------
    def submit(self, rid, stream, kind, count, arrival=None):
        """Queue a request; returns it with status "waiting", or "rejected" when it is
        larger than the arena or would push the waiting bytes past max_queued_bytes."""
        r = Request(rid, int(stream), int(kind), int(count), self.now() if arrival is None else arrival)
        r.nbytes = r.count * (8 if r.kind == KIND_F64 else 4)
        held = -(-max(r.nbytes, 1) // _ALIGN) * _ALIGN     # what the arena would reserve
        if held > self.arena.size or (self.max_queued_bytes is not None and
                                          self.queued_bytes + r.nbytes > self.max_queued_bytes):
            r.status = "rejected"
            self.rejected.append(r)
            return r
        b, p = self.cur_block[r.stream], self.cur_pos[r.stream]
        r.skip, r.pos = b, p
        self.cur_block[r.stream], self.cur_pos[r.stream] = advance_cursor(b, p, r.kind, r.count)
        self.queued_bytes += r.nbytes
        self.pending[r.rid] = r
        self.waiting.append(r)
        return r

    def cancel(self, rid):
        """Cancel a request that has not been launched; returns False if it has (or is
        unknown).  Its arena block, if any, is released at once."""
        r = self.pending.pop(rid, None)
        if r is None:
            return False
        if r.status == "waiting":
            self.waiting.remove(r)
            self.queued_bytes -= r.nbytes
        else:
            self.admitted.remove(r)
            self.arena.release(r.offset, r.reserved)
        r.status = "cancelled"
        self.cancelled.append(r)
        return True

    def _admit(self):
        while self.waiting:
            r = self.waiting[0]
            got = self.arena.alloc(max(r.nbytes, 1))
            if got is None:
                return
            r.offset, r.reserved = got
            self.waiting.popleft()
            self.queued_bytes -= r.nbytes
            r.status = "admitted"
            self.admitted.append(r)

    def _dispatch(self):
        torch = self.torch
        while self.admitted and self.free_streams:
            batch = [self.admitted.popleft() for _ in range(min(self.max_batch, len(self.admitted)))]
            si = self.free_streams.popleft()
            st = self.streams[si]
            reqs = np.zeros(len(batch), dtype=B.request_dtype())
            reqs["stream"] = [r.stream for r in batch]
            reqs["skip"] = [r.skip for r in batch]
            reqs["pos"] = [r.pos for r in batch]
            reqs["kind"] = [r.kind for r in batch]
            reqs["count"] = [r.count for r in batch]
            reqs["offset"] = [r.offset // (8 if r.kind == KIND_F64 else 4) for r in batch]
            base = self.dev.data_ptr()
            groups = []   # (event, requests): each request completes with its group's event
            with torch.cuda.stream(st):
                B.rlxpp_draw_requests(self.gen.handle, reqs, base, base, 0, st)
                if self.host is not None:
                    # small requests first, one copy per run of adjacent arena blocks, so
                    # that they do not wait behind the large copies of the same batch;
                    # then each large request by itself, smallest first
                    small = [r for r in batch if r.nbytes < self.small_bytes]
                    large = sorted((r for r in batch if r.nbytes >= self.small_bytes), key=lambda r: r.nbytes)
                    if small:
                        spans = sorted((r.offset, r.reserved) for r in small if r.nbytes)
                        k = 0
                        while k < len(spans):
                            a, ln = spans[k]
                            while k + 1 < len(spans) and spans[k + 1][0] == a + ln:
                                ln += spans[k + 1][1]
                                k += 1
                            self.host[a:a + ln].copy_(self.dev[a:a + ln], non_blocking=True)
                            k += 1
                        ev = torch.cuda.Event()
                        ev.record(st)
                        groups.append((ev, small))
                    for r in large:
                        self.host[r.offset:r.offset + r.nbytes].copy_(self.dev[r.offset:r.offset + r.nbytes],
                                                                     non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(st)
                        groups.append((ev, [r]))
                else:
                    ev = torch.cuda.Event()
                    ev.record(st)
                    groups.append((ev, batch))
            t = self.now()
            for r in batch:
                r.launch = t
                r.status = "launched"
                self.pending.pop(r.rid, None)
            self.inflight.append((si, collections.deque(groups)))

    def _complete(self, wait_first=False):
        """Retire every request whose copy has finished (any order); a CUDA stream is
        free again once its batch's last group is done.  Optionally wait for the
        oldest batch's next group first."""
        if wait_first and self.inflight:
            self.inflight[0][1][0][0].synchronize()
        keep = collections.deque()
        while self.inflight:
            si, groups = self.inflight.popleft()
            while groups and groups[0][0].query():  # a stream's groups finish in order
                _, done = groups.popleft()
                t = self.now()
                for r in done:
                    r.done = t
                    r.status = "done"
                    if self.keep_results and self.host is not None and r.nbytes:
                        raw = self.host[r.offset:r.offset + r.nbytes].numpy()
                        r.result = raw.view(np.uint64 if r.kind == KIND_F64 else np.uint32).copy()
                    self.arena.release(r.offset, r.reserved)
                    self.finished.append(r)
            if groups:
                keep.append((si, groups))
            else:
                self.free_streams.append(si)
        self.inflight = keep

    def pump(self):
        """One round: complete finished batches, admit, launch."""
        self._complete()
        self._admit()
        self._dispatch()

    def drain(self):
        """Run everything submitted so far to completion."""
        while self.waiting or self.admitted or self.inflight:
            self.pump()
            if self.inflight and (not self.free_streams or not self.admitted):
                self._complete(wait_first=True)

    def close(self):
        self.torch.cuda.synchronize()
        self.gen.close()

    # -- trace replay ---------------------------------------------------------------------
    def run_trace(self, arrival_s, stream, count, is_f64, duration=None):
        """Release requests at their (wall-clock) arrival times; returns stats.  Python's
        cyclic garbage collector is paused meanwhile: its full passes over the many live
        request objects would stall the loop and every request in flight with it."""
        n = len(arrival_s)
        if duration is not None:
            n = int(np.searchsorted(arrival_s, duration))
        was_enabled = gc.isenabled()
        gc.disable()
        try:
            self.t0 = time.perf_counter()
            i = 0
            while i < n or self.waiting or self.admitted or self.inflight:
                t = self.now()
                while i < n and arrival_s[i] <= t:
                    self.submit(i, stream[i], KIND_F64 if is_f64[i] else KIND_U24, count[i],
                                arrival=float(arrival_s[i]))
                    i += 1
                self.pump()
                if i < n and not self.admitted and not self.waiting:
                    gap = arrival_s[i] - self.now()
                    if gap > 2e-4 and not self.inflight:
                        time.sleep(min(gap, 1e-3))
            self.torch.cuda.synchronize()
        finally:
            if was_enabled:
                gc.enable()
        return self.stats()

    def stats(self):
        if not self.finished:
            return {}
        lat = np.array([r.done - r.arrival for r in self.finished])
        first = min(r.arrival for r in self.finished)
        last = max(r.done for r in self.finished)
        values = sum(r.count for r in self.finished)
        doubles = sum(r.count for r in self.finished if r.kind == KIND_F64)
        return {"requests": len(self.finished), "rejected": len(self.rejected), "cancelled": len(self.cancelled),
                "values": values, "doubles": doubles,
                "seconds": last - first, "values_per_s": values / (last - first),
                "doubles_per_s": doubles / (last - first),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3)}


class NativeServer:
    """The same serving loop with the host side in the library (rlxpp_server_*): no
    Python runs per request.  Results and records as for Server: take_done() returns the
    completed requests (numpy records of struct rlxpp_served), result(rec) a kept result
    (keep_results=True), run_trace() the latency of every request of a trace."""

    def __init__(self, n_resident, luxury=2048, seeds=None, pool_bytes=1 << 30, n_cuda_streams=4,
                 max_batch=512, keep_results=False, copy_to_host=True, small_bytes=1 << 20,
                 max_queued_bytes=None):
        import torch
        if seeds is None:
            seeds = np.arange(1, n_resident + 1, dtype=np.uint64)
        self.gen = B.Generator(n_resident, [luxury], torch.from_numpy(np.asarray(seeds, np.uint64).view(np.int64)).cuda())
        flags = (B.RLXPP_SERVER_COPY_TO_HOST if copy_to_host else 0) | (B.RLXPP_SERVER_KEEP_RESULTS if keep_results else 0)
        self.handle = B.rlxpp_server_create(self.gen.handle, pool_bytes, n_cuda_streams, max_batch, small_bytes,
                                            max_queued_bytes or 0, flags)

    def submit(self, rid, stream, kind, count, arrival=-1.0):
        """True if accepted (False: rejected by the admission bound)."""
        return B.rlxpp_server_submit(self.handle, rid, stream, kind, count, arrival)

    def cancel(self, rid):
        return B.rlxpp_server_cancel(self.handle, rid)

    def pump(self, wait=False):
        B.rlxpp_server_pump(self.handle, wait)

    def drain(self):
        B.rlxpp_server_drain(self.handle)

    def stats(self):
        return B.rlxpp_server_stats(self.handle)

    def take_done(self):
        return B.rlxpp_server_take_done(self.handle)

    def result(self, rec):
        out = np.zeros(int(rec["count"]), dtype=np.uint64 if rec["kind"] == KIND_F64 else np.uint32)
        B.rlxpp_server_result(self.handle, int(rec["rid"]), out)
        return out

    def run_trace(self, arrival_s, stream, count, is_f64):
        return B.rlxpp_server_run_trace(self.handle, arrival_s, stream, count, is_f64)

    def close(self):
        self.torch_sync()
        B.rlxpp_server_destroy(self.handle)
        self.gen.close()

    @staticmethod
    def torch_sync():
        import torch
        torch.cuda.synchronize()
