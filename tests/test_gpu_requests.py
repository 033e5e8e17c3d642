"""Batched requests (rlxpp_plan_requests / rlxpp_run_plan / rlxpp_draw_requests) against
the oracle, bit-exact (GPU): uneven counts, mixed kinds and luxury levels, skips,
arbitrary start positions, the same stream several times, chunking by jump-ahead at
several chunk lengths, RLXPP_REQ_ADVANCE, CUDA-graph capture of a run (one kernel node
for all luxury levels), the tuner, and the single-stream workload (2^20 doubles from
seed 1) split over many threads; on the three request kernels (one thread per chunk on
the integer pipe or on the tensor cores, one warp per chunk)."""
import numpy as np
import pytest

from oracle import ranluxpp as R
from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import StreamSet, seeded_X

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(params=["tensor", "imad", "warp"])
def path(request):
    return request.param


def path_id(native, path):
    return {"imad": native.RLXPP_PATH_IMAD, "tensor": native.RLXPP_PATH_TENSOR, "warp": native.RLXPP_PATH_WARP}[path]


def set_path(native, g, path):
    g.set_path(path_id(native, path))


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def expected(X, p, skip, pos, kind, count):
    """Oracle: the stream at LCG state X, skipped by `skip` advances, read from `pos`."""
    Xs = pow(R.luxury_multiplier(p), skip, R.M) * X % R.M
    ss = StreamSet([Xs], p, pos=[pos])
    out = ss.draw(count, S.KIND_F64 if kind == 1 else S.KIND_U24)[0]
    return (out.view(np.uint64) if kind == 1 else out), ss


def make_requests(rows):
    import paper_2106_02504_gb300._rlxpp as B
    a = np.zeros(len(rows), dtype=B.request_dtype())
    for i, (stream, skip, pos, kind, count) in enumerate(rows):
        a[i] = (stream, skip, pos, kind, count, 0)
    off = {0: 0, 1: 0}
    for i in range(len(a)):
        k = int(a[i]["kind"])
        a[i]["offset"] = off[k]
        off[k] += int(a[i]["count"])
    return a, off[0], off[1]


def run_and_check(native, g, xs, levels_of, reqs, n_u24, n_f64, flags=0, tuning=None, graph=False):
    out_u = torch.full((max(n_u24, 1),), -1, dtype=torch.int32, device="cuda")
    out_f = torch.full((max(n_f64, 1),), -1, dtype=torch.int64, device="cuda")
    plan = native.rlxpp_plan_requests(g.handle, reqs, flags, tuning)
    try:
        if graph:
            cg = torch.cuda.CUDAGraph()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                native.rlxpp_run_plan(g.handle, plan, out_u, out_f, s)   # warm-up outside capture
            torch.cuda.current_stream().wait_stream(s)
            out_u.fill_(-1)
            out_f.fill_(-1)
            with torch.cuda.graph(cg):
                native.rlxpp_run_plan(g.handle, plan, out_u, out_f)
            cg.replay()
            cg.replay()
        else:
            native.rlxpp_run_plan(g.handle, plan, out_u, out_f)
        torch.cuda.synchronize()
        items = native.rlxpp_plan_items(plan)
    finally:
        native.rlxpp_destroy_plan(plan)
    gu = out_u.cpu().numpy().view(np.uint32)
    gf = out_f.cpu().numpy().view(np.uint64)
    finals = {}
    for r in reqs:
        st, skip, pos, kind, count, off = (int(r[k]) for k in ("stream", "skip", "pos", "kind", "count", "offset"))
        want, ss = expected(xs[st], levels_of[st], skip, pos, kind, count)
        got = gf[off:off + count] if kind == 1 else gu[off:off + count]
        assert np.array_equal(got, want), (st, skip, pos, kind, count)
        finals[st] = ss.state_records()[0]
    return items, finals


def current_X(native, g, n):
    buf = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    g.get_state(buf)
    rec = buf.cpu().numpy().view(np.uint64)
    xs = []
    for i in range(n):
        D = sum(int(rec[i, k]) << (64 * k) for k in range(9))
        xs.append(R.to_lcg(D, int(rec[i, 9]) & 1))
    return xs, rec


def test_mixed_requests(native, path):
    n = 200
    levels = [24, 223, 389, 2048]
    lvl = (np.arange(n) % 4).astype(np.uint8)
    seeds = W.random_seeds(n, 201)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(),
                         torch.from_numpy(lvl).cuda())
    set_path(native, g, path)
    xs, _ = current_X(native, g, n)
    levels_of = [levels[int(lvl[i])] for i in range(n)]
    rng = np.random.Generator(np.random.PCG64(202))
    rows = []
    for i in range(300):
        st = int(rng.integers(0, n))
        skip = int(rng.choice([0, 0, 1, 5, int(rng.integers(0, 2 ** 40)), 2 ** 63]))
        pos = int(rng.integers(0, 25))
        kind = int(rng.integers(0, 2))
        count = int(rng.choice([0, 1, 2, 11, 12, 13, 24, 25, int(rng.integers(0, 3000))]))
        rows.append((st, skip, pos, kind, count))
    reqs, nu, nf = make_requests(rows)
    for tuning in [(2, 2), (4, 4), (64, 3), (16, 2, (native.rlxpp_get_path(g.handle) + 1) % 3), None]:
        run_and_check(native, g, xs, levels_of, reqs, nu, nf, tuning=tuning)
    # streams did not move
    xs2, _ = current_X(native, g, n)
    assert xs2 == xs


def test_block_shapes(native):
    """Every block shape the tuner tries (64, 128, 256 threads per CTA on the integer
    kernels, 128 on the tensor kernel) gives the oracle's values at mixed levels; shapes
    outside them are refused when planning."""
    n = 150
    levels = [24, 389, 2048]
    lvl = (np.arange(n) % 3).astype(np.uint8)
    seeds = W.random_seeds(n, 211)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(),
                         torch.from_numpy(lvl).cuda())
    xs, _ = current_X(native, g, n)
    levels_of = [levels[int(lvl[i])] for i in range(n)]
    rng = np.random.Generator(np.random.PCG64(212))
    rows = [(i, int(rng.integers(0, 2 ** 20)), int(rng.integers(0, 25)), int(rng.integers(0, 2)),
             int(rng.integers(0, 4000))) for i in range(n)]
    reqs, nu, nf = make_requests(rows)
    I, T, Wp = native.RLXPP_PATH_IMAD, native.RLXPP_PATH_TENSOR, native.RLXPP_PATH_WARP
    for tuning in [(8, 4, I, 64), (8, 8, I, 64), (8, 1, I, 256), (8, 2, I, 256), (8, 3, T, 128),
                   (8, 4, Wp, 64), (8, 2, Wp, 128), (8, 1, Wp, 256), (8, 2, Wp, 256)]:
        run_and_check(native, g, xs, levels_of, reqs, nu, nf, tuning=tuning)
    for bad in [(8, 2, T, 64), (8, 2, T, 256), (8, 2, I, 96), (8, 2, I, 512), (8, 8, I, 512)]:
        with pytest.raises(native.RlxppError):
            native.rlxpp_plan_requests(g.handle, reqs, 0, bad)


def test_advance_flag_and_graph(native, path):
    n = 130
    seeds = W.consecutive_seeds(n, first=300)
    g = native.Generator(n, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    set_path(native, g, path)
    xs, _ = current_X(native, g, n)
    rng = np.random.Generator(np.random.PCG64(203))
    rows = [(i, int(rng.integers(0, 1000)), int(rng.integers(0, 25)), int(rng.integers(0, 2)),
             int(rng.integers(0, 5000))) for i in range(n)]
    rows[0] = (0, 7, 3, 1, 0)      # count 0: only the skip and position move the stream
    reqs, nu, nf = make_requests(rows)
    _, finals = run_and_check(native, g, xs, [2048] * n, reqs, nu, nf, flags=native.RLXPP_REQ_ADVANCE,
                              tuning=(8, 2))
    buf = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    g.get_state(buf)
    rec = buf.cpu().numpy().view(np.uint64)
    for st, want in finals.items():
        assert np.array_equal(rec[st], want), st
    # graph-captured run of a plan without ADVANCE, replayed twice: same values
    xs, _ = current_X(native, g, n)
    rows = [(i, 0, 0, i % 2, 777) for i in range(n)]
    reqs, nu, nf = make_requests(rows)
    run_and_check(native, g, xs, [2048] * n, reqs, nu, nf, tuning=(16, 3), graph=True)


def test_strided_chunks(native):
    """Tensor path: requests of at least 32 L blocks after their start block go out as
    warps of 32 strided chunks (lane t draws blocks f + t, f + t + 32, ... by products
    with A^32).  Counts that end exactly at a warp's last block (the request's last block
    then in lane 31), one block, a partial block and a warp past it; start positions that
    leave a head or none; skips; u24 and f64 at odd and even output offsets (runs that
    start 4-, 8- and 16-byte aligned); at L = 12 also remainders of hundreds of blocks;
    every value against the oracle and, with RLXPP_REQ_ADVANCE, every final state."""
    n = 48
    levels = [24, 389, 2048]
    lvl = (np.arange(n) % 3).astype(np.uint8)
    seeds = W.random_seeds(n, 205)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(),
                         torch.from_numpy(lvl).cuda())
    g.set_path(native.RLXPP_PATH_TENSOR)
    levels_of = [levels[int(lvl[i])] for i in range(n)]
    for L in (2, 3, 12):
        xs, _ = current_X(native, g, n)
        rows = []
        for i in range(n):
            kind = i % 2
            per = 12 if kind else 24
            pos = [0, 24, 2, 7, 23][i % 5] & (~1 if kind else ~0)  # f64 heads start on even words
            room = (24 - pos) // (2 if kind else 1)
            nb = 32 * L * (1 + i % 3) + [0, 1, 256, 33, 32 * L - 1, 300][(i // 3) % 6]
            count = room + (nb - 1) * per + [per, per, per - 5, 1, per // 2][(i // 5) % 5]
            rows.append((i, [0, 3, 1000][i % 3], pos, kind, count))
        reqs, nu, nf = make_requests(rows)
        _, finals = run_and_check(native, g, xs, levels_of, reqs, nu, nf, flags=native.RLXPP_REQ_ADVANCE,
                                  tuning=(L, 2, native.RLXPP_PATH_TENSOR, 128))
        buf = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
        g.get_state(buf)
        rec = buf.cpu().numpy().view(np.uint64)
        for st, want in finals.items():
            assert np.array_equal(rec[st], want), (L, st)


def test_chunking_matches_plain_draw(native, path):
    """One long request split at several chunk lengths equals rlxpp_draw_f64."""
    seeds = np.array([42, 43], dtype=np.uint64)
    count = 100_003
    ref = native.Generator(2, [389], torch.from_numpy(seeds.view(np.int64)).cuda())
    plain = torch.zeros((2, count), dtype=torch.float64, device="cuda")
    ref.draw_f64(plain, count)
    g = native.Generator(2, [389], torch.from_numpy(seeds.view(np.int64)).cuda())
    set_path(native, g, path)
    import paper_2106_02504_gb300._rlxpp as B
    reqs = np.zeros(2, dtype=B.request_dtype())
    reqs[0] = (0, 0, 0, 1, count, 0)
    reqs[1] = (1, 0, 0, 1, count, count)
    for L in (2, 3, 16, 1000):
        out = torch.zeros(2 * count, dtype=torch.float64, device="cuda")
        plan = native.rlxpp_plan_requests(g.handle, reqs, 0, (L, 3))
        native.rlxpp_run_plan(g.handle, plan, None, out)
        torch.cuda.synchronize()
        native.rlxpp_destroy_plan(plan)
        assert torch.equal(out.view(2, count), plain), L


def test_single_stream_split(native, path):
    """Seed 1, p = 2048, 2^20 doubles drawn by many threads through jump-ahead."""
    n = 1 << 20
    g = native.Generator(1, [2048], torch.ones(1, dtype=torch.int64, device="cuda"))
    set_path(native, g, path)
    import paper_2106_02504_gb300._rlxpp as B
    reqs = np.zeros(1, dtype=B.request_dtype())
    reqs[0] = (0, 0, 0, 1, n, 0)
    out = torch.zeros(n, dtype=torch.float64, device="cuda")
    plan = native.rlxpp_plan_requests(g.handle, reqs, native.RLXPP_REQ_ADVANCE)
    assert native.rlxpp_plan_items(plan) > 1000
    native.rlxpp_run_plan(g.handle, plan, None, out)
    torch.cuda.synchronize()
    native.rlxpp_destroy_plan(plan)
    ref = StreamSet.from_seeds([1], 2048)
    want = ref.draw(n, S.KIND_F64).view(np.uint64)[0]
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)
    buf = torch.zeros((1, 11), dtype=torch.int64, device="cuda")
    g.get_state(buf)
    assert np.array_equal(buf.cpu().numpy().view(np.uint64)[0], ref.state_records()[0])


def test_autotune(native, path):
    n = 512
    seeds = W.consecutive_seeds(n)
    g = native.Generator(n, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    set_path(native, g, path)
    xs, _ = current_X(native, g, n)
    counts = W.log_uniform_counts(n, 1, 20000, seed=204)
    rows = [(i, 0, 0, i % 2, int(counts[i])) for i in range(n)]
    reqs, nu, nf = make_requests(rows)
    out_u = torch.zeros(max(nu, 1), dtype=torch.int32, device="cuda")
    out_f = torch.zeros(max(nf, 1), dtype=torch.float64, device="cuda")
    best = native.rlxpp_autotune_requests(g.handle, reqs, out_u, out_f)
    assert best[0] >= 2 and 1 <= best[1] <= 8 and best[2] in (0, 1, 2) and best[3] in (64, 128, 256)
    assert best[1] * best[3] <= 2048 and (best[2] != native.RLXPP_PATH_TENSOR or best[3] == 128)
    plan = native.rlxpp_plan_requests(g.handle, reqs)        # uses the tuned choice
    assert native.rlxpp_plan_tuning(plan) == best
    native.rlxpp_destroy_plan(plan)
    run_and_check(native, g, xs, [2048] * n, reqs, nu, nf)


def test_tune_cache_file(native, tmp_path, monkeypatch):
    """RLXPP_TUNE_CACHE: the tuner appends its choice (with the block shape) and a later
    handle plans with it; a line without the block shape still reads (default shape)."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("RLXPP_TUNE_CACHE", str(cache))
    n = 256
    seeds = torch.from_numpy(W.consecutive_seeds(n).view(np.int64)).cuda()
    rows = [(i, 0, 0, i % 2, 3000 + i) for i in range(n)]
    reqs, nu, nf = make_requests(rows)
    out_u = torch.zeros(max(nu, 1), dtype=torch.int32, device="cuda")
    out_f = torch.zeros(max(nf, 1), dtype=torch.float64, device="cuda")
    g = native.Generator(n, [2048], seeds)
    best = native.rlxpp_autotune_requests(g.handle, reqs, out_u, out_f)
    g.close()
    line = cache.read_text().strip().splitlines()[-1].split("|")
    assert len(line) == 6 and tuple(int(v) for v in line[2:]) == best
    g2 = native.Generator(n, [2048], seeds)
    plan = native.rlxpp_plan_requests(g2.handle, reqs)
    assert native.rlxpp_plan_tuning(plan) == best
    native.rlxpp_destroy_plan(plan)
    g2.close()
    # a line in the older five-field form, for the same shape, wins (later lines win)
    with open(cache, "a") as f:
        f.write("|".join(line[:2] + ["8", "3", str(native.RLXPP_PATH_IMAD)]) + "\n")
    g3 = native.Generator(n, [2048], seeds)
    xs, _ = current_X(native, g3, n)
    plan = native.rlxpp_plan_requests(g3.handle, reqs)
    assert native.rlxpp_plan_tuning(plan) == (8, 3, native.RLXPP_PATH_IMAD, 0)
    native.rlxpp_destroy_plan(plan)
    run_and_check(native, g3, xs, [2048] * n, reqs, nu, nf)
    g3.close()


def _captured_node_types(fn, stream):
    """Node types of the CUDA graph that capturing fn() on `stream` records (driver API:
    0 kernel, 1 memcpy, 2 memset, ...)."""
    import ctypes
    cu = ctypes.CDLL("libcuda.so.1")
    begin = getattr(cu, "cuStreamBeginCapture_v2", None) or cu.cuStreamBeginCapture
    graph = ctypes.c_void_p()
    assert begin(ctypes.c_void_p(stream.cuda_stream), 2) == 0   # CU_STREAM_CAPTURE_MODE_RELAXED
    try:
        fn()
    finally:
        assert cu.cuStreamEndCapture(ctypes.c_void_p(stream.cuda_stream), ctypes.byref(graph)) == 0
    try:
        n = ctypes.c_size_t(0)
        assert cu.cuGraphGetNodes(graph, None, ctypes.byref(n)) == 0
        nodes = (ctypes.c_void_p * max(n.value, 1))()
        assert cu.cuGraphGetNodes(graph, nodes, ctypes.byref(n)) == 0
        types = []
        for k in range(n.value):
            t = ctypes.c_int(-1)
            assert cu.cuGraphNodeGetType(ctypes.c_void_p(nodes[k]), ctypes.byref(t)) == 0
            types.append(t.value)
        return types
    finally:
        cu.cuGraphDestroy(graph)


def test_one_kernel_node_for_all_levels(native, path):
    """A run of a plan over four luxury levels, captured on a stream, is one kernel node
    (no per-level launches and no memset: the work counters reset themselves), and two
    runs after the capture give the oracle's values."""
    n = 96
    levels = [24, 223, 389, 2048]
    lvl = (np.arange(n) % 4).astype(np.uint8)
    seeds = W.consecutive_seeds(n, first=900)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(), torch.from_numpy(lvl).cuda())
    xs, _ = current_X(native, g, n)
    rows = [(i, i * 3, i % 25, i % 2, 50 + 37 * i) for i in range(n)]
    reqs, nu, nf = make_requests(rows)
    out_u = torch.full((nu,), -1, dtype=torch.int32, device="cuda")
    out_f = torch.full((nf,), -1, dtype=torch.int64, device="cuda")
    plan = native.rlxpp_plan_requests(g.handle, reqs, 0, (4, 2, path_id(native, path)))
    try:
        s = torch.cuda.Stream()
        torch.cuda.synchronize()
        types = _captured_node_types(lambda: native.rlxpp_run_plan(g.handle, plan, out_u, out_f, s), s)
        assert types == [0], types
        for _ in range(2):
            native.rlxpp_run_plan(g.handle, plan, out_u, out_f, s)
        torch.cuda.synchronize()
    finally:
        native.rlxpp_destroy_plan(plan)
    gu = out_u.cpu().numpy().view(np.uint32)
    gf = out_f.cpu().numpy().view(np.uint64)
    for r in reqs:
        st, skip, pos, kind, count, off = (int(r[k]) for k in ("stream", "skip", "pos", "kind", "count", "offset"))
        want, _ = expected(xs[st], levels[int(lvl[st])], skip, pos, kind, count)
        got = gf[off:off + count] if kind == 1 else gu[off:off + count]
        assert np.array_equal(got, want), (st, kind, count)


def test_request_validation(native):
    g = native.Generator(4, [24], torch.arange(1, 5, dtype=torch.int64, device="cuda"))
    import paper_2106_02504_gb300._rlxpp as B
    for row in [(4, 0, 0, 0, 1), (0, 0, 25, 0, 1), (0, 0, 0, 2, 1), (0, 0, 0, 0, -1)]:
        reqs = np.zeros(1, dtype=B.request_dtype())
        reqs[0] = (*row, 0)
        with pytest.raises(native.RlxppError):
            native.rlxpp_plan_requests(g.handle, reqs)
    reqs = np.zeros(2, dtype=B.request_dtype())
    reqs[0] = (1, 0, 0, 0, 5, 0)
    reqs[1] = (1, 9, 0, 0, 5, 5)
    native.rlxpp_destroy_plan(native.rlxpp_plan_requests(g.handle, reqs))   # fine without ADVANCE
    with pytest.raises(native.RlxppError):
        native.rlxpp_plan_requests(g.handle, reqs, native.RLXPP_REQ_ADVANCE)
    with pytest.raises(native.RlxppError):
        native.rlxpp_plan_requests(g.handle, reqs, 0, (1, 4))                # chunk length < 2
    plan = native.rlxpp_plan_requests(g.handle, np.zeros(0, dtype=B.request_dtype()))
    native.rlxpp_run_plan(g.handle, plan)
    native.rlxpp_destroy_plan(plan)
