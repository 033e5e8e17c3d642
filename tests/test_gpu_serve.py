"""The continuous-batching loop (GPU): a Poisson trace through a small device arena (so
requests wait for memory), several CUDA streams and small batches; every result must
equal the same request run alone, and each stream's results, in arrival order, must
equal the oracle's sequence for that stream (mixed u24 and f64 draws)."""
import numpy as np
import pytest

from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import StreamSet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def test_serving_results_alone_and_in_mix(native):
    from paper_2106_02504_gb300.serve import Server
    n_res = 300
    arr, stream, counts, is_f64 = W.serving_trace(400, rate_hz=4000, n_resident=n_res, lo=100, hi=20000, seed=5)
    srv = Server(n_res, pool_bytes=1 << 20, n_cuda_streams=3, max_batch=16, keep_results=True)
    stats = srv.run_trace(arr, stream, counts, is_f64)
    assert stats["requests"] == 400 and stats["p99_ms"] >= stats["p50_ms"] > 0
    seeds = np.arange(1, n_res + 1, dtype=np.uint64)
    g = native.Generator(n_res, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    import paper_2106_02504_gb300._rlxpp as B
    for r in srv.finished:
        req = np.zeros(1, dtype=B.request_dtype())
        req[0] = (r.stream, r.skip, r.pos, r.kind, r.count, 0)
        dt = torch.float64 if r.kind == 1 else torch.int32
        out = torch.zeros(max(r.count, 1), dtype=dt, device="cuda")
        native.rlxpp_draw_requests(g.handle, req, None if r.kind == 1 else out, out if r.kind == 1 else None)
        alone = out.cpu().numpy().view(np.uint64 if r.kind == 1 else np.uint32)[:r.count]
        assert np.array_equal(alone, r.result), r.rid
    # per-stream sequences against the oracle, for the streams with the most requests
    by_stream = {}
    for r in sorted(srv.finished, key=lambda r: r.rid):
        by_stream.setdefault(r.stream, []).append(r)
    busiest = sorted(by_stream, key=lambda s: -len(by_stream[s]))[:6]
    for s in busiest:
        ss = StreamSet.from_seeds([s + 1], 2048)
        for r in by_stream[s]:
            want = ss.draw(r.count, S.KIND_F64 if r.kind == 1 else S.KIND_U24)[0]
            assert np.array_equal(r.result, want.view(np.uint64) if r.kind == 1 else want), (s, r.rid)
    srv.close()
    g.close()


def _stream_reference(stream, requests):
    """The oracle's values for one stream's requests in submission order, each drawn
    whether or not it ran (a cancelled request's segment is skipped, not reused)."""
    ref = StreamSet.from_seeds([stream + 1], 2048)
    out = {}
    for r in requests:
        vals = ref.draw(r.count, S.KIND_F64 if r.kind == 1 else S.KIND_U24)[0]
        out[r.rid] = vals.view(np.uint64) if r.kind == 1 else vals
    return out


def test_admission_rejects_without_taking_stream_numbers(native):
    """A bound on the bytes waiting for the arena: requests past it, and one larger than
    the whole arena, are rejected at submission; the accepted requests of each stream
    still read its sequence without a gap."""
    from paper_2106_02504_gb300.serve import Server
    srv = Server(4, pool_bytes=1 << 16, n_cuda_streams=2, max_batch=4, keep_results=True,
                 max_queued_bytes=40_000)
    rng = np.random.Generator(np.random.PCG64(11))
    subs = []
    for rid in range(24):        # submitted before any pumping: the queue fills up
        stream, kind, count = int(rng.integers(0, 4)), int(rng.integers(0, 2)), int(rng.integers(1, 2500))
        subs.append(srv.submit(rid, stream, kind, count))
    big = srv.submit(99, 0, 1, 10_000)       # 80,000 bytes: more than the arena
    assert big.status == "rejected"
    rejected = [r for r in subs if r.status == "rejected"]
    accepted = [r for r in subs if r.status == "waiting"]
    assert rejected and accepted and sum(r.nbytes for r in accepted) <= 40_000
    srv.drain()
    # after the queue drained, a request is accepted again
    late = srv.submit(100, 1, 0, 500)
    assert late.status == "waiting"
    srv.drain()
    stats = srv.stats()
    assert stats["rejected"] == len(rejected) + 1 and stats["requests"] == len(accepted) + 1
    done = accepted + [late]
    assert all(r.status == "done" for r in done) and all(r.result is None for r in rejected)
    for s in range(4):
        mine = [r for r in done if r.stream == s]
        want = _stream_reference(s, mine)
        for r in mine:
            assert np.array_equal(r.result, want[r.rid]), (s, r.rid)
    srv.close()


def test_cancel_before_launch(native):
    """Requests cancelled while waiting for the arena or admitted but not launched are
    dropped (their arena block released at once) and their segments skipped; a launched
    request cannot be cancelled; the rest equal the oracle."""
    from paper_2106_02504_gb300.serve import Server
    srv = Server(2, pool_bytes=1 << 15, n_cuda_streams=1, max_batch=1, keep_results=True)
    reqs = [srv.submit(rid, rid % 2, rid % 2, 600 + 50 * rid) for rid in range(8)]
    assert srv.cancel(1)                        # waiting
    srv.pump()                                  # admits what fits, launches one batch of one
    launched = [r for r in reqs if r.status == "launched"]
    admitted = [r for r in reqs if r.status == "admitted"]
    assert len(launched) == 1 and admitted
    assert not srv.cancel(launched[0].rid)
    used = srv.arena.used
    victim = admitted[-1]
    assert srv.cancel(victim.rid) and srv.arena.used == used - victim.reserved
    assert not srv.cancel(victim.rid) and not srv.cancel(12345)
    srv.drain()
    cancelled = {1, victim.rid}
    assert {r.rid for r in srv.cancelled} == cancelled and srv.stats()["cancelled"] == 2
    for s in range(2):
        mine = [r for r in reqs if r.stream == s]
        want = _stream_reference(s, mine)
        for r in mine:
            if r.rid in cancelled:
                assert r.status == "cancelled" and r.result is None
            else:
                assert r.status == "done" and np.array_equal(r.result, want[r.rid]), r.rid
    srv.close()


def _segments(stream, kind, count):
    """(skip, pos) of each request by the cursor rule, in submission order."""
    from paper_2106_02504_gb300.serve import advance_cursor
    cur = {}
    out = []
    for s, k, c in zip(stream, kind, count):
        b, p = cur.get(int(s), (0, 0))
        out.append((b, p))
        cur[int(s)] = advance_cursor(b, p, int(k), int(c))
    return out


def test_native_serving_trace_matches_oracle(native):
    """The library's serving loop on a Poisson trace through a small arena (requests
    wait for memory), three CUDA streams and small batches: every kept result equals the
    oracle's values for its stream segment, and each stream read in request order is the
    oracle's sequence."""
    from paper_2106_02504_gb300.serve import NativeServer
    n_res = 300
    arr, stream, counts, is_f64 = W.serving_trace(400, rate_hz=4000, n_resident=n_res, lo=100, hi=20000, seed=7)
    srv = NativeServer(n_res, pool_bytes=1 << 20, n_cuda_streams=3, max_batch=16, keep_results=True)
    lat = srv.run_trace(arr, stream, counts, is_f64)
    st = srv.stats()
    assert np.all(lat > 0) and st["done"] == 400
    # every batch's device times were read: the request kernel and the copies took time,
    # and no batch's device time exceeds the longest request latency
    assert st["batches_timed"] >= 400 // 16 and st["kernel_us_sum"] > 0 and st["copy_us_sum"] > 0
    assert st["kernel_us_max"] + st["copy_us_max"] <= 1e6 * float(lat.max()) + 1000
    kinds = is_f64.astype(int)
    by_stream = {}
    seeds = np.arange(1, n_res + 1, dtype=np.uint64)
    g = native.Generator(n_res, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    for i, ((s, k, c), (skip, pos)) in enumerate(zip(zip(stream, kinds, counts), _segments(stream, kinds, counts))):
        rec = np.zeros(1, dtype=native.served_dtype())[0]
        rec["rid"], rec["kind"], rec["count"] = i, k, c
        got = srv.result(rec)
        # the same request alone
        req = np.zeros(1, dtype=native.request_dtype())
        req[0] = (s, skip, pos, k, c, 0)
        out = torch.zeros(max(int(c), 1), dtype=torch.float64 if k else torch.int32, device="cuda")
        native.rlxpp_draw_requests(g.handle, req, None if k else out, out if k else None)
        alone = out.cpu().numpy().view(np.uint64 if k else np.uint32)[:c]
        assert np.array_equal(alone, got), i
        by_stream.setdefault(int(s), []).append((k, int(c), got))
    g.close()
    for s, items in by_stream.items():
        ref = StreamSet.from_seeds([s + 1], 2048)
        for k, c, got in items:
            want = ref.draw(c, S.KIND_F64 if k else S.KIND_U24)[0]
            assert np.array_equal(got, want.view(np.uint64) if k else want), s
    srv.close()


def test_native_admission_and_cancel(native):
    """Admission bound: rejected requests take no stream numbers; cancellation while
    waiting or admitted skips the segment and frees the arena block; a launched request
    cannot be cancelled; the served results equal the oracle."""
    from paper_2106_02504_gb300.serve import NativeServer
    srv = NativeServer(4, pool_bytes=1 << 16, n_cuda_streams=2, max_batch=4, keep_results=True,
                       max_queued_bytes=40_000)
    rng = np.random.Generator(np.random.PCG64(11))
    subs = []
    for rid in range(24):
        s, k, c = int(rng.integers(0, 4)), int(rng.integers(0, 2)), int(rng.integers(1, 2500))
        subs.append((rid, s, k, c, srv.submit(rid, s, k, c)))
    assert not srv.submit(99, 0, 1, 10_000)                  # larger than the arena
    accepted = [x for x in subs if x[4]]
    assert accepted and len(accepted) < len(subs)
    assert srv.stats()["rejected"] == len(subs) - len(accepted) + 1
    srv.drain()
    recs = {int(r["rid"]): r for r in srv.take_done()}
    assert set(recs) == {x[0] for x in accepted}
    for s in range(4):
        ref = StreamSet.from_seeds([s + 1], 2048)
        for rid, s2, k, c, _ in accepted:
            if s2 != s:
                continue
            want = ref.draw(c, S.KIND_F64 if k else S.KIND_U24)[0]
            assert np.array_equal(srv.result(recs[rid]), want.view(np.uint64) if k else want), rid
    srv.close()

    # a pool of 1000 bytes holds three 256-byte granules: 960 bytes (1024 once rounded)
    # are refused at once rather than waiting forever
    srv = NativeServer(2, pool_bytes=1000, n_cuda_streams=1, max_batch=1)
    assert not srv.submit(0, 0, 0, 240) and srv.submit(1, 0, 0, 192)
    srv.drain()
    assert [int(r["rid"]) for r in srv.take_done()] == [1]
    srv.close()

    srv = NativeServer(2, pool_bytes=1 << 15, n_cuda_streams=1, max_batch=1, keep_results=True)
    reqs = [(rid, rid % 2, rid % 2, 600 + 50 * rid) for rid in range(8)]
    for rid, s, k, c in reqs:
        assert srv.submit(rid, s, k, c)
    assert srv.cancel(1)                                      # waiting
    srv.pump()                                                # admits what fits, launches request 0
    st = srv.stats()
    assert st["admitted"] >= 1 and st["inflight_groups"] >= 1
    assert not srv.cancel(0)                                  # launched
    used = st["arena_used"]
    assert srv.cancel(2) and srv.stats()["arena_used"] < used  # admitted: its block is freed
    assert not srv.cancel(2) and not srv.cancel(12345)
    srv.drain()
    recs = {int(r["rid"]): r for r in srv.take_done()}
    assert set(recs) == {0, 3, 4, 5, 6, 7} and srv.stats()["cancelled"] == 2
    for s in range(2):
        ref = StreamSet.from_seeds([s + 1], 2048)
        for rid, s2, k, c in reqs:
            if s2 != s:
                continue
            want = ref.draw(c, S.KIND_F64 if k else S.KIND_U24)[0]   # cancelled segments skipped
            if rid in recs:
                assert np.array_equal(srv.result(recs[rid]), want.view(np.uint64) if k else want), rid
    srv.close()
