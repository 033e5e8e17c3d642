"""Full-size parity on every stream, in exactly the launch configurations bench.py times.

* The 2^20-stream step (seed, 1024 doubles per stream into an 8 GiB device buffer, 4096
  more into the exact sum and 256-bin histogram) on both refill paths: every stream's
  1024 doubles (by a position-weighted 64-bit checksum per stream, which any single
  changed value alters), every stream's sum, the whole histogram bin by bin and every
  final state, against the C recurrence oracle run over all 2^20 streams.
* The 65,536-stream mixed batch with the tuner's own plan (rlxpp_autotune_requests, as
  bench.py calls it), captured in a CUDA graph and replayed, on both product kernels:
  every request's values by the same checksum, against the oracle stream by stream.
* The 2^18 uniform 128-bit skips followed by 48 doubles: every stream's doubles and
  final state against pow(A, n, m) (a spawned process pool computes the powers)."""
import multiprocessing
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import (StreamSet, records_from_windows, seeded_X, skipped_states,
                               weighted_checksum)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 1 << 20
P = 2048
HBM, FUSED = 1024, 4096
CHUNK = 1 << 16


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P_
    return P_.native


def _cores():
    return S.default_threads()


@pytest.fixture(scope="module")
def step_oracle():
    """The oracle's view of one benchmark step over all 2^20 streams: per-stream
    checksums of the 1024 doubles, per-stream sums of the 4096 fused doubles, the whole
    histogram and every final state record."""
    seeds = W.consecutive_seeds(N)
    xs = seeded_X(seeds, P)
    cks = np.zeros(N, dtype=np.uint64)
    sums = np.zeros(N, dtype=np.uint64)
    hist = np.zeros(256, dtype=np.uint64)
    recs = np.zeros((N, 11), dtype=np.uint64)
    for a in range(0, N, CHUNK):
        ss = StreamSet([xs[int(s)] for s in seeds[a:a + CHUNK]], P)
        cks[a:a + CHUNK] = weighted_checksum(ss.draw(HBM, S.KIND_F64).view(np.uint64))
        s_, h_ = ss.sum_hist(FUSED)
        sums[a:a + CHUNK] = s_
        hist += h_
        recs[a:a + CHUNK] = records_from_windows(ss.words, ss.carry, ss.pos, P)
    return seeds, cks, sums, hist, recs


def _device_checksums(out):
    """weighted_checksum of every row of a (rows, cols) int64 device tensor, in chunks."""
    w = torch.arange(1, 2 * out.shape[1], 2, dtype=torch.int64, device=out.device)
    res = torch.empty(out.shape[0], dtype=torch.int64, device=out.device)
    for a in range(0, out.shape[0], CHUNK):
        res[a:a + CHUNK] = (out[a:a + CHUNK] * w).sum(dim=1)
    return res.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("path", ["tensor", "imad"])
def test_bench_step_every_stream_full_size(native, step_oracle, path):
    seeds, cks, wsums, whist, wrecs = step_oracle
    seeds_d = torch.from_numpy(seeds.view(np.int64)).cuda()
    g = native.Generator(N, [P], seeds_d)
    g.set_path(native.RLXPP_PATH_TENSOR if path == "tensor" else native.RLXPP_PATH_IMAD)
    out = torch.empty((N, HBM), dtype=torch.float64, device="cuda")
    sums = torch.zeros(N, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.seed(seeds_d)                               # one step as bench.py runs it
    g.draw_f64(out, HBM)
    g.draw_f64_sum_hist(FUSED, sums, hist)
    st = torch.zeros((N, 11), dtype=torch.int64, device="cuda")
    g.get_state(st)
    g.sync()
    got = _device_checksums(out.view(torch.int64))
    bad = np.nonzero(got != cks)[0]
    assert bad.size == 0, f"{bad.size} streams' doubles differ, first {bad[:5]}"
    bad = np.nonzero(sums.cpu().numpy().view(np.uint64) != wsums)[0]
    assert bad.size == 0, f"{bad.size} streams' sums differ, first {bad[:5]}"
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), whist)
    bad = np.nonzero((st.cpu().numpy().view(np.uint64) != wrecs).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} final states differ, first {bad[:5]}"
    del out
    g.close()


def _request_checksum_oracle(seed, p, count, f64):
    ss = StreamSet.from_seeds([seed], p)
    v = ss.draw(count, S.KIND_F64 if f64 else S.KIND_U24)[0]
    return weighted_checksum(v.view(np.uint64) if f64 else v)


@pytest.fixture(scope="module")
def batch_oracle():
    levels, lvl, counts, is_f64 = W.batch_mix(65536, seed=3)
    seeds = np.arange(1, 65537, dtype=np.uint64)
    order = np.argsort(-counts)       # longest first keeps the pool busy to the end
    want = np.zeros(65536, dtype=np.uint64)

    def one(i):
        want[i] = _request_checksum_oracle(int(seeds[i]), levels[int(lvl[i])], int(counts[i]), bool(is_f64[i]))

    with ThreadPoolExecutor(_cores()) as ex:
        list(ex.map(one, order.tolist()))
    return levels, lvl, counts, is_f64, seeds, want


@pytest.mark.parametrize("path", ["tensor", "imad"])
def test_config3_tuned_plan_every_request(native, batch_oracle, path):
    """The tuner's (chunk length, blocks per SM) with each product kernel, as bench.py
    replays it from a CUDA graph; every request's values against the oracle."""
    import paper_2106_02504_gb300._rlxpp as B
    levels, lvl, counts, is_f64, seeds, want = batch_oracle
    n = len(seeds)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(), torch.from_numpy(lvl).cuda())
    kind = is_f64.astype(np.uint32)
    off = np.zeros(n, dtype=np.int64)
    for k in (0, 1):
        sel = kind == k
        off[sel] = np.concatenate([[0], np.cumsum(counts[sel])[:-1]])
    reqs = np.zeros(n, dtype=B.request_dtype())
    reqs["stream"] = np.arange(n)
    reqs["kind"] = kind
    reqs["count"] = counts
    reqs["offset"] = off
    nf, nu = int(counts[is_f64].sum()), int(counts[~is_f64].sum())
    out_f = torch.full((nf + 1,), -1, dtype=torch.int64, device="cuda")
    out_u = torch.full((nu + 1,), -1, dtype=torch.int32, device="cuda")
    tuned = native.rlxpp_autotune_requests(g.handle, reqs, out_u, out_f)
    pid = native.RLXPP_PATH_TENSOR if path == "tensor" else native.RLXPP_PATH_IMAD
    plan = native.rlxpp_plan_requests(g.handle, reqs, 0, (tuned[0], tuned[1], pid, tuned[3] if pid == tuned[2] else 0))
    st = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(st)
    with torch.cuda.stream(side):       # the warm-up run bench.py makes before capturing
        native.rlxpp_run_plan(g.handle, plan, out_u, out_f, side.cuda_stream)
    st.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        native.rlxpp_run_plan(g.handle, plan, out_u, out_f)
    out_f.fill_(-1)
    out_u.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    native.rlxpp_destroy_plan(plan)
    assert int(out_f[-1]) == -1 and int(out_u[-1]) == -1            # nothing past the outputs
    w = torch.arange(1, 2 * int(counts.max()) + 1, 2, dtype=torch.int64, device="cuda")
    got = torch.empty(n, dtype=torch.int64, device="cuda")
    for i in range(n):
        o, c = int(off[i]), int(counts[i])
        src = out_f[o:o + c] if is_f64[i] else out_u[o:o + c].to(torch.int64)
        got[i] = (src * w[:c]).sum()
    got = got.cpu().numpy().view(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} requests differ, first {bad[:5]}"
    del graph
    g.close()


def test_config4_every_stream_full_size(native):
    """2^18 streams (seeds i + 1, p = 2048) skipped by uniform 128-bit distances, then 48
    doubles each, as bench.py times it: every stream's doubles and final state."""
    n = 1 << 18
    seeds = W.consecutive_seeds(n)
    dist = W.skip_distances(n, seed=4)
    xs = seeded_X(seeds, P)
    pairs = [(xs[int(seeds[i])], int(dist[i, 0]) | (int(dist[i, 1]) << 64)) for i in range(n)]
    jobs = [(P, pairs[a:a + 4096]) for a in range(0, n, 4096)]
    # the pool is spawned (never forked from a process that already uses CUDA)
    with multiprocessing.get_context("spawn").Pool(_cores()) as pool:
        Xs = [x for part in pool.map(skipped_states, jobs) for x in part]
    g = native.Generator(n, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.skip(torch.from_numpy(dist.view(np.int64)).cuda())
    out = torch.empty((n, 48), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 48)
    st = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    g.get_state(st)
    g.sync()
    ref = StreamSet(Xs, P)
    want = ref.draw(48, S.KIND_F64).view(np.uint64)
    got = out.cpu().numpy().view(np.uint64)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} streams' doubles differ, first {bad[:5]}"
    wrec = records_from_windows(ref.words, ref.carry, ref.pos, P)
    bad = np.nonzero((st.cpu().numpy().view(np.uint64) != wrec).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} final states differ, first {bad[:5]}"
    g.close()
