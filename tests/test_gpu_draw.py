"""Generator entry points against the oracle, element by element, bit-exact (GPU).

Seeding, skipping, u24/f64 draws (uniform and ragged per-stream counts, odd read
positions, host and device outputs), the fused sum/histogram consumer, state export /
import and its validation, mixed luxury levels, and the single-stream workload
(2^20 doubles and 2^20 integers from seed 1 at p = 2048; 10,000 advances at p = 24)."""
import numpy as np
import pytest

from oracle import ranluxpp as R
from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import StreamSet, normals_expected, exponentials_expected, from_limbs64, seeded_X

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def dev_u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def states(native, g, n):
    buf = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    native.rlxpp_get_state(g.handle, buf)
    return buf.cpu().numpy().view(np.uint64)


def assert_states(native, g, ref: StreamSet):
    n = ref.words.shape[0]
    got = states(native, g, n)
    want = ref.state_records()
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} streams differ, first {bad[:5]}"


def f64_bits(t):
    return t.cpu().numpy().view(np.uint64)


N = 300  # three blocks of 128 threads and a ragged tail


@pytest.fixture(params=["tensor", "imad", "warp"])
def path(request):
    return request.param


def path_id(native, path):
    return {"imad": native.RLXPP_PATH_IMAD, "tensor": native.RLXPP_PATH_TENSOR, "warp": native.RLXPP_PATH_WARP}[path]


def make(native, seeds, levels=(2048,), level_of=None, path=None):
    lo = None if level_of is None else torch.from_numpy(np.asarray(level_of, dtype=np.uint8)).cuda()
    g = native.Generator(len(seeds), list(levels), dev_u64(seeds), lo)
    if path is not None and (len(levels) == 1 or path == "warp"):
        g.set_path(path_id(native, path))
    return g


def test_seed_states(native):
    seeds = W.consecutive_seeds(N)
    g = make(native, seeds)
    assert_states(native, g, StreamSet.from_seeds(seeds, 2048))
    # extreme seeds: the smallest, 2^63 and the largest
    seeds2 = np.array([1, 2, 2 ** 63, 2 ** 64 - 1, 2718, 123456789012345], dtype=np.uint64)
    g2 = make(native, seeds2, levels=(389,))
    assert_states(native, g2, StreamSet.from_seeds(seeds2, 389))
    g.close()
    g2.close()


def _seed_records(seeds, levels, level_of):
    rec = np.zeros((len(seeds), 11), dtype=np.uint64)
    for i, s in enumerate(seeds):
        p = levels[level_of[i]]
        D, c = R.to_ranlux(R.seed_lcg(int(s), p))
        rec[i, :9] = [(D >> (64 * k)) & (2 ** 64 - 1) for k in range(9)]
        rec[i, 9] = c
        rec[i, 10] = p
    return rec


def test_seed_runs(native):
    """Seeding continues a run of consecutive seeds at one level by one product per stream:
    runs that cross the kernel's groups of 8 streams, broken runs, repeated and
    descending seeds, the largest seeds, level changes inside a run and a ragged tail, on
    a new handle and when re-seeding, against the oracle."""
    seeds = list(range(1, 20)) + [100, 101, 103, 104, 2 ** 64 - 2, 2 ** 64 - 1, 1, 2, 7, 7, 8, 5, 4] + \
        list(range(1000, 1037))
    seeds = np.array(seeds, dtype=np.uint64)
    n = len(seeds)
    levels = (24, 2048)
    level_of = [(i // 5) % 2 for i in range(n)]   # a level change every 5 streams
    g = make(native, seeds, levels=levels, level_of=level_of)
    assert np.array_equal(states(native, g, n), _seed_records(seeds, levels, level_of))
    re = seeds + np.uint64(5)                       # re-seed: the same runs, shifted
    re[re < 5] = 9                                  # (2^64 - 2 and 2^64 - 1 wrapped)
    g.seed(dev_u64(re))
    assert np.array_equal(states(native, g, n), _seed_records(re, levels, level_of))
    g.sync()


def test_zero_seed_rejected(native):
    """Seeds start at 1: a zero in a host array fails the call at once; a zero in a
    device array is reported by rlxpp_sync, a re-seeded stream with seed 0 keeps its
    state and the other streams are seeded as usual."""
    seeds = np.array([5, 0, 7], dtype=np.uint64)
    with pytest.raises(native.RlxppError) as e:
        native.Generator(3, [2048], torch.from_numpy(seeds.view(np.int64)))      # host seeds
    assert e.value.status == native.RLXPP_ERR_INVALID
    g = make(native, np.array([5, 6, 7], dtype=np.uint64))
    with pytest.raises(native.RlxppError):
        g.seed(torch.from_numpy(seeds.view(np.int64)))                             # host seeds
    assert_states(native, g, StreamSet.from_seeds([5, 6, 7], 2048))               # nothing moved
    g.seed(dev_u64(np.array([9, 0, 11], dtype=np.uint64)))                        # device seeds
    with pytest.raises(native.RlxppError) as e:
        g.sync()
    assert e.value.status == native.RLXPP_ERR_INVALID
    assert_states(native, g, StreamSet.from_seeds([9, 6, 11], 2048))             # stream 1 kept
    g.sync()                                                                       # cleared
    g.close()


@pytest.mark.parametrize("p,count", [(2048, 1000), (24, 1001), (223, 12), (389, 1)])
def test_draw_f64_uniform(native, p, count, path):
    seeds = W.random_seeds(N, 31 + p)
    g = make(native, seeds, levels=(p,), path=path)
    out = torch.zeros((N, count), dtype=torch.float64, device="cuda")
    g.draw_f64(out, count)
    ref = StreamSet.from_seeds(seeds, p)
    want = ref.draw(count, S.KIND_F64)
    assert np.array_equal(f64_bits(out), want.view(np.uint64))
    assert_states(native, g, ref)


@pytest.mark.parametrize("p,count", [(2048, 1000), (24, 24), (389, 23)])
def test_draw_u24_uniform(native, p, count, path):
    seeds = W.random_seeds(N, 41 + p)
    g = make(native, seeds, levels=(p,), path=path)
    out = torch.zeros((N, count), dtype=torch.int32, device="cuda")
    g.draw_u24(out, count)
    ref = StreamSet.from_seeds(seeds, p)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), ref.draw(count, S.KIND_U24))
    assert_states(native, g, ref)


def test_mixed_types_odd_positions(native, path):
    """u24 draws leave odd read positions; doubles then skip a lone leftover word."""
    seeds = W.consecutive_seeds(N, first=77)
    g = make(native, seeds, levels=(223,), path=path)
    ref = StreamSet.from_seeds(seeds, 223)
    for kind, count in [(S.KIND_U24, 5), (S.KIND_F64, 7), (S.KIND_U24, 23), (S.KIND_F64, 30),
                        (S.KIND_U24, 1), (S.KIND_F64, 11), (S.KIND_F64, 0), (S.KIND_U24, 48)]:
        if kind == S.KIND_U24:
            out = torch.zeros((N, max(count, 1)), dtype=torch.int32, device="cuda")
            g.draw_u24(out, count)
            got = out.cpu().numpy().view(np.uint32)[:, :count]
        else:
            out = torch.zeros((N, max(count, 1)), dtype=torch.float64, device="cuda")
            g.draw_f64(out, count)
            got = f64_bits(out)[:, :count]
        want = ref.draw(count, kind)
        if kind == S.KIND_F64:
            want = want.view(np.uint64)
        assert np.array_equal(got, want), (kind, count)
    assert_states(native, g, ref)


def _draw(native, g, kind, count, n):
    dt = {S.KIND_U24: torch.int32, S.KIND_F64: torch.float64, S.KIND_F32: torch.float32}[kind]
    out = torch.full((n, max(count, 1)), -1, dtype=dt, device="cuda")
    {S.KIND_U24: g.draw_u24, S.KIND_F64: g.draw_f64, S.KIND_F32: g.draw_f32}[kind](out, count)
    a = out.cpu().numpy()[:, :count]
    return a.view(np.uint64) if kind == S.KIND_F64 else a.view(np.uint32)


def _want(ref, kind, count):
    w = ref.draw(count, kind)
    return w.view(np.uint64) if kind == S.KIND_F64 else w.view(np.uint32)


def test_tile_stores_heads_and_tails(native, path):
    """Uniform draws whose blocks go out as one store per tile when the tile's streams
    move in step: fresh blocks, heads that keep the first column 16-byte aligned and
    heads that do not, counts whose row length is or is not a multiple of 16 bytes,
    ragged last blocks and a ragged last tile; then positions that differ within a
    tile (a ragged draw first)."""
    seeds = W.random_seeds(N, 91)
    g = make(native, seeds, levels=(389,), path=path)
    ref = StreamSet.from_seeds(seeds, 389)
    steps = [(S.KIND_F64, 996), (S.KIND_U24, 4), (S.KIND_F64, 1000), (S.KIND_U24, 2), (S.KIND_F64, 998),
             (S.KIND_F32, 100), (S.KIND_U24, 3), (S.KIND_F32, 1001), (S.KIND_F32, 96), (S.KIND_U24, 1),
             (S.KIND_F64, 26), (S.KIND_U24, 500), (S.KIND_F64, 1002)]
    for kind, count in steps:
        assert np.array_equal(_draw(native, g, kind, count, N), _want(ref, kind, count)), (kind, count)
    assert_states(native, g, ref)
    # streams at different positions inside each tile, then uniform draws again
    counts, offsets = W.ragged_counts(N, 30, seed=92)
    out = torch.zeros(int(counts.sum()) + 1, dtype=torch.int32, device="cuda")
    g.draw_u24(out, 0, torch.from_numpy(counts).cuda(), torch.from_numpy(offsets).cuda())
    got = out.cpu().numpy().view(np.uint32)
    for i, w in enumerate(ref.draw_ragged(counts, S.KIND_U24)):
        assert np.array_equal(got[offsets[i]:offsets[i] + counts[i]], w), i
    for kind, count in [(S.KIND_F64, 1000), (S.KIND_U24, 96), (S.KIND_F32, 48)]:
        assert np.array_equal(_draw(native, g, kind, count, N), _want(ref, kind, count)), (kind, count)
    assert_states(native, g, ref)
    g.close()


def test_draw_normal(native, path):
    """Gaussian values (Box-Muller on consecutive pairs of doubles) against the oracle
    within the derived tolerance; odd counts, starts inside a block, ragged counts, a
    host output buffer; the streams end where the f64 draw of 2 ceil(n / 2) values
    leaves them."""
    seeds = W.random_seeds(N, 93)
    g = make(native, seeds, levels=(389,), path=path)
    ref = StreamSet.from_seeds(seeds, 389)
    for kind, count, host in [("n", 1000, False), (S.KIND_U24, 3, False), ("n", 1001, False), (S.KIND_F64, 5, False),
                              ("n", 7, True), ("n", 1, False), ("n", 0, False)]:
        if kind != "n":
            _draw(native, g, kind, count, N)
            ref.draw(count, kind)
            continue
        out = torch.full((N, max(count, 1)), 7.0, dtype=torch.float64, device="cpu" if host else "cuda")
        g.draw_normal_f64(out, count)
        got = out.cpu().numpy()[:, :count]
        want, tol = normals_expected(ref.draw(count + (count & 1), S.KIND_F64), count)
        assert np.all(np.abs(got - want) <= tol), (count, float(np.max(np.abs(got - want) - tol)))
        if count == 0:
            assert np.all(out.cpu().numpy() == 7.0)
    assert_states(native, g, ref)
    # ragged counts (odd and even) into one packed output
    counts, offsets = W.ragged_counts(N, 41, seed=94)
    out = torch.full((int(counts.sum()) + 1,), 7.0, dtype=torch.float64, device="cuda")
    g.draw_normal_f64(out, 0, torch.from_numpy(counts).cuda(), torch.from_numpy(offsets).cuda())
    got = out.cpu().numpy()
    for i, d in enumerate(ref.draw_ragged(counts + (counts & 1), S.KIND_F64)):
        c = int(counts[i])
        if c == 0:
            continue
        want, tol = normals_expected(d.reshape(1, -1), c)
        assert np.all(np.abs(got[offsets[i]:offsets[i] + c] - want[0]) <= tol[0]), i
    assert got[-1] == 7.0
    assert_states(native, g, ref)
    g.close()


def test_draw_exp(native, path):
    """Exponential values (inversion, one double each) against the oracle within the
    derived tolerance; starts inside a block, ragged counts, a host output buffer; the
    streams end where the f64 draw of the same count leaves them."""
    seeds = W.random_seeds(N, 95)
    g = make(native, seeds, levels=(223,), path=path)
    ref = StreamSet.from_seeds(seeds, 223)
    for kind, count, host in [("e", 1000, False), (S.KIND_U24, 3, False), ("e", 1001, False),
                              ("e", 5, True), ("e", 1, False), ("e", 0, False)]:
        if kind != "e":
            _draw(native, g, kind, count, N)
            ref.draw(count, kind)
            continue
        out = torch.full((N, max(count, 1)), 7.0, dtype=torch.float64, device="cpu" if host else "cuda")
        g.draw_exp_f64(out, count)
        got = out.cpu().numpy()[:, :count]
        want, tol = exponentials_expected(ref.draw(count, S.KIND_F64))
        assert np.all(np.abs(got - want) <= tol), (count, float(np.max(np.abs(got - want) - tol)))
        assert np.all(got >= 0)
        if count == 0:
            assert np.all(out.cpu().numpy() == 7.0)
    assert_states(native, g, ref)
    counts, offsets = W.ragged_counts(N, 41, seed=96)
    out = torch.full((int(counts.sum()) + 1,), 7.0, dtype=torch.float64, device="cuda")
    g.draw_exp_f64(out, 0, torch.from_numpy(counts).cuda(), torch.from_numpy(offsets).cuda())
    got = out.cpu().numpy()
    for i, d in enumerate(ref.draw_ragged(counts, S.KIND_F64)):
        c = int(counts[i])
        want, tol = exponentials_expected(d)
        assert np.all(np.abs(got[offsets[i]:offsets[i] + c] - want) <= tol), i
    assert got[-1] == 7.0
    assert_states(native, g, ref)
    g.close()


def test_warp_path_single_stream(native):
    """One stream read in order on the warp path (one warp per stream): 100,001 doubles,
    then 50,001 u24 and 777 f32, every value and the final state against the oracle."""
    g = make(native, np.array([1], dtype=np.uint64), path="warp")
    ref = StreamSet.from_seeds([1], 2048)
    for kind, count in [(S.KIND_F64, 100001), (S.KIND_U24, 50001), (S.KIND_F32, 777)]:
        assert np.array_equal(_draw(native, g, kind, count, 1), _want(ref, kind, count)), kind
    assert_states(native, g, ref)
    g.close()


@pytest.mark.parametrize("kind", [S.KIND_U24, S.KIND_F64])
def test_ragged_counts_offsets(native, kind, path):
    seeds = W.random_seeds(N, 51)
    counts, offsets = W.ragged_counts(N, 200, seed=52)
    total = int(counts.sum())
    g = make(native, seeds, levels=(2048,), path=path)
    dt = torch.int32 if kind == S.KIND_U24 else torch.float64
    out = torch.full((total + 1,), -1, dtype=dt, device="cuda")
    c_d = torch.from_numpy(counts).cuda()
    o_d = torch.from_numpy(offsets).cuda()
    (g.draw_u24 if kind == S.KIND_U24 else g.draw_f64)(out, 0, c_d, o_d)
    got = out.cpu().numpy()
    ref = StreamSet.from_seeds(seeds, 2048)
    for i in range(N):
        one = StreamSet.__new__(StreamSet)
        one.p, one.words, one.carry, one.pos = 2048, ref.words[i:i + 1], ref.carry[i:i + 1], ref.pos[i:i + 1]
        w = one.draw(int(counts[i]), kind)[0]
        seg = got[offsets[i]:offsets[i] + counts[i]]
        if kind == S.KIND_F64:
            assert np.array_equal(seg.view(np.uint64), w.view(np.uint64)), i
        else:
            assert np.array_equal(seg.view(np.uint32), w), i
    assert got[total] == -1  # nothing written past the packed output
    assert_states(native, g, ref)


def test_sum_hist(native, path):
    seeds = W.consecutive_seeds(N, first=1000)
    g = make(native, seeds, levels=(2048,), path=path)
    sums = torch.zeros(N, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(4096, sums, hist)
    ref = StreamSet.from_seeds(seeds, 2048)
    wsums, whist = ref.sum_hist(4096)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), wsums)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), whist)
    assert int(hist.sum()) == N * 4096
    # accumulation across calls, with a ragged count
    g.draw_f64_sum_hist(13, sums, hist)
    wsums2, whist2 = ref.sum_hist(13)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), wsums2)  # sums are overwritten
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), whist + whist2)
    assert_states(native, g, ref)


@pytest.mark.parametrize("p", [24, 223, 389, 2048])
def test_sum_hist_levels_and_positions(native, p, path):
    """The fused consumer at the four mixed-batch levels (the tensor path's matrix for
    operand rows that hold the RANLUX numbers, with its block-sum columns, is built per
    level) from streams left at every read position by a ragged u24 draw, with a count
    that ends in a partial block; sums, histogram and final states against the oracle."""
    seeds = W.random_seeds(N, 77 + p)
    g = make(native, seeds, levels=(p,), path=path)
    counts = (np.arange(N) * 7) % 29
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    out = torch.zeros(int(counts.sum()) + 1, dtype=torch.int32, device="cuda")
    g.draw_u24(out, 0, torch.from_numpy(counts.astype(np.int64)).cuda(), torch.from_numpy(offs).cuda())
    sums = torch.zeros(N, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(1001, sums, hist)
    ref = StreamSet.from_seeds(seeds, p)
    ref.draw_ragged(counts, S.KIND_U24)
    wsums, whist = ref.sum_hist(1001)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), wsums)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), whist)
    assert_states(native, g, ref)


def test_skip(native):
    seeds = W.consecutive_seeds(N)
    p = 2048
    g = make(native, seeds, levels=(p,))
    # move some streams off position 0 first
    out = torch.zeros((N, 5), dtype=torch.int32, device="cuda")
    g.draw_u24(out, 5)
    dist = W.skip_distances(N, seed=4)
    dist[0] = [0, 0]
    dist[1] = [1, 0]
    dist[2] = [2 ** 64 - 1, 2 ** 64 - 1]
    g.skip(dev_u64(dist))
    xs = seeded_X(seeds, p)
    A = R.luxury_multiplier(p)
    got = states(native, g, N)
    for i in range(N):
        n = int(dist[i, 0]) | (int(dist[i, 1]) << 64)
        X = pow(A, n, R.M) * xs[int(seeds[i])] % R.M
        D, c = R.to_ranlux(X)
        assert from_limbs64(got[i, :9]) == D, i
        assert int(got[i, 9]) == c | (5 << 32), i


def test_state_round_trip_and_validation(native):
    seeds = W.random_seeds(N, 61)
    g = make(native, seeds, levels=(24, 2048), level_of=np.arange(N) % 2)
    out1 = torch.zeros((N, 50), dtype=torch.float64, device="cuda")
    g.draw_f64(out1, 50)
    saved = states(native, g, N).copy()
    out2 = torch.zeros((N, 77), dtype=torch.float64, device="cuda")
    g.draw_f64(out2, 77)
    # restore from host memory and draw again: same numbers
    g.set_state(saved.view(np.int64).copy())
    g.sync()
    out3 = torch.zeros((N, 77), dtype=torch.float64, device="cuda")
    g.draw_f64(out3, 77)
    assert torch.equal(out2, out3)
    # a host copy of the state continues the same sequence (Sec. 4.2)
    assert np.array_equal(states(native, g, N)[:, 10], np.where(np.arange(N) % 2, 2048, 24))
    # invalid records: bad carry, bad pos, unknown p, non-canonical numbers, zero state
    bad = states(native, g, N).copy()
    keep = bad.copy()
    bad[0, 9] = 2                                   # carry 2
    bad[1, 9] = 25 << 32                            # pos 25
    bad[2, 10] = 7                                  # p not a level of the handle
    bad[3, :9] = 0
    bad[3, 9] = 0                                   # X = 0
    bad[4, :9] = [2 ** 64 - 1] * 9
    bad[4, 9] = 1                                   # X = m
    g.set_state(bad.view(np.int64).copy())
    with pytest.raises(native.RlxppError) as e:
        g.sync()
    assert e.value.status == native.RLXPP_ERR_INVALID
    got = states(native, g, N)
    assert np.array_equal(got[:5], keep[:5])        # rejected streams unchanged
    assert np.array_equal(got[5:], bad[5:])
    g.sync()                                        # status was cleared


def test_noncanonical_record_rejected(native):
    # find a non-canonical (D, c): to_ranlux(to_lcg(D, c)) != (D, c)
    rng = np.random.Generator(np.random.PCG64(71))
    for _ in range(100):
        w = [int(x) for x in rng.integers(0, 2 ** 24, size=24)]
        c = int(rng.integers(0, 2))
        X = R.to_lcg(R.pack_words(w), c)
        if 0 < X < R.M and R.to_ranlux(X) != (R.pack_words(w), c):
            break
    g = make(native, np.array([5], dtype=np.uint64), levels=(2048,))
    rec = states(native, g, 1).copy()
    D = R.pack_words(w)
    rec[0, :9] = [(D >> (64 * k)) & (2 ** 64 - 1) for k in range(9)]
    rec[0, 9] = c
    g.set_state(rec.view(np.int64).copy())
    with pytest.raises(native.RlxppError):
        g.sync()


def test_mixed_levels(native, path):
    # per-stream multipliers: the integer kernel for the tensor path (its tiles share one
    # level), the warp kernel's per-level loads for the warp path
    levels, lvl_idx, _, _ = W.batch_mix(N, seed=81)
    seeds = W.random_seeds(N, 82)
    g = make(native, seeds, levels=levels, level_of=lvl_idx, path=path)
    out = torch.zeros((N, 40), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 40)
    got = f64_bits(out)
    refs = []
    for li, p in enumerate(levels):
        idx = np.nonzero(lvl_idx == li)[0]
        ref = StreamSet.from_seeds(seeds[idx], p)
        assert np.array_equal(got[idx], ref.draw(40, S.KIND_F64).view(np.uint64)), p
        refs.append((idx, ref))
    # the fused consumer, then u24, on the same handle
    sums = torch.zeros(N, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(300, sums, hist)
    out_u = torch.zeros((N, 30), dtype=torch.int32, device="cuda")
    g.draw_u24(out_u, 30)
    gs = sums.cpu().numpy().view(np.uint64)
    gu = out_u.cpu().numpy().view(np.uint32)
    for idx, ref in refs:
        ws, _ = ref.sum_hist(300)
        assert np.array_equal(gs[idx], ws)
        assert np.array_equal(gu[idx], ref.draw(30, S.KIND_U24))
    assert int(hist.sum()) == N * 300
    g.close()


def test_reseed(native):
    g = make(native, W.consecutive_seeds(N), levels=(24, 389), level_of=np.arange(N) % 2)
    out = torch.zeros((N, 9), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 9)
    seeds = W.random_seeds(N, 91)
    g.seed(dev_u64(seeds))
    g.draw_f64(out, 9)
    got = f64_bits(out)
    for li, p in enumerate((24, 389)):
        idx = np.nonzero(np.arange(N) % 2 == li)[0]
        assert np.array_equal(got[idx], StreamSet.from_seeds(seeds[idx], p).draw(9, S.KIND_F64).view(np.uint64))


def test_host_buffers(native):
    """Pageable and pinned host outputs and host inputs (seeds, counts, offsets)."""
    seeds = W.random_seeds(N, 101)
    g = native.Generator(N, [2048], seeds)            # seeds from pageable host memory
    h = np.zeros((N, 100), dtype=np.float64)
    g.draw_f64(h, 100)                                # pageable host output
    ref = StreamSet.from_seeds(seeds, 2048)
    assert np.array_equal(h.view(np.uint64), ref.draw(100, S.KIND_F64).view(np.uint64))
    pinned = torch.zeros((N, 64), dtype=torch.int32).pin_memory()
    g.draw_u24(pinned, 64)
    assert np.array_equal(pinned.numpy().view(np.uint32), ref.draw(64, S.KIND_U24))
    counts, offsets = W.ragged_counts(N, 30, seed=102)
    hc = np.zeros(int(counts.sum()), dtype=np.float64)
    g.draw_f64(hc, 0, counts, offsets)                # host counts/offsets/output
    for i in range(0, N, 37):
        one = StreamSet.__new__(StreamSet)
        one.p, one.words, one.carry, one.pos = 2048, ref.words[i:i + 1], ref.carry[i:i + 1], ref.pos[i:i + 1]
        want = one.draw(int(counts[i]), S.KIND_F64)[0]
        assert np.array_equal(hc[offsets[i]:offsets[i] + counts[i]].view(np.uint64), want.view(np.uint64))


def test_host_output_chunked(native):
    """Host output larger than one device staging chunk (256 MiB): 2^16 streams x 1024."""
    n, count = 1 << 16, 1024
    seeds = W.consecutive_seeds(n)
    g = make(native, seeds)
    h = torch.zeros((n, count), dtype=torch.float64).pin_memory()
    g.draw_f64(h, count)
    d = torch.zeros((n, count), dtype=torch.float64, device="cuda")
    g2 = make(native, seeds)
    g2.draw_f64(d, count)
    assert torch.equal(h, d.cpu())
    idx = [0, 1, 4095, 4096, n - 1]
    ref = StreamSet.from_seeds(seeds[idx], 2048)
    assert np.array_equal(h.numpy()[idx].view(np.uint64), ref.draw(count, S.KIND_F64).view(np.uint64))


def test_empty_and_zero(native):
    g = native.Generator(0, [2048], None)
    assert native.rlxpp_num_streams(g.handle) == 0
    g.draw_f64(None, 0)
    g.sync()
    g1 = make(native, W.consecutive_seeds(3))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    g1.draw_f64(out, 0)
    with pytest.raises(native.RlxppError):
        native.rlxpp_draw_f64(g1.handle, out, -1)
    with pytest.raises(native.RlxppError):
        native.rlxpp_create(1, [0], np.array([1], dtype=np.uint64))


def test_single_stream_workload(native, path):
    """Seed 1, p = 2048: 2^20 doubles, and 2^20 integers from a fresh seed-1 state."""
    n = 1 << 20
    for kind in (S.KIND_F64, S.KIND_U24):
        g = make(native, np.array([1], dtype=np.uint64), path=path)
        dt = torch.float64 if kind == S.KIND_F64 else torch.int32
        out = torch.zeros((1, n), dtype=dt, device="cuda")
        (g.draw_f64 if kind == S.KIND_F64 else g.draw_u24)(out, n)
        ref = StreamSet.from_seeds([1], 2048)
        want = ref.draw(n, kind)
        got = out.cpu().numpy()
        if kind == S.KIND_F64:
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        else:
            assert np.array_equal(got.view(np.uint32), want)
        assert_states(native, g, ref)


def test_p24_ten_thousand_advances(native, path):
    """10,000 refills at p = 24 on one stream, each block equal to 24 recurrence steps."""
    g = make(native, np.array([1], dtype=np.uint64), levels=(24,), path=path)
    n = 24 * 10_001
    out = torch.zeros((1, n), dtype=torch.int32, device="cuda")
    g.draw_u24(out, n)
    got = out.cpu().numpy().view(np.uint32)[0]
    w, c = R.to_ranlux(R.seed_lcg(1, 24))
    w = R.unpack_words(w)
    for b in range(10_001):
        assert list(got[24 * b:24 * (b + 1)]) == w, b
        w, c = S.block(w, c, 24)


@pytest.mark.parametrize("p,count", [(2048, 1000), (24, 25)])
def test_draw_f32(native, p, count, path):
    seeds = W.random_seeds(N, 111 + p)
    g = make(native, seeds, levels=(p,), path=path)
    g.draw_u24(torch.zeros((N, 3), dtype=torch.int32, device="cuda"), 3)   # odd positions
    out = torch.zeros((N, count), dtype=torch.float32, device="cuda")
    g.draw_f32(out, count)
    ref = StreamSet.from_seeds(seeds, p)
    ref.draw(3, S.KIND_U24)
    want = ref.draw(count, S.KIND_F32)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want.view(np.uint32))
    assert_states(native, g, ref)


@pytest.mark.parametrize("kind,need", [(0, 1), (1, 2), (2, 1)])
def test_skip_values(native, kind, need):
    p = 389
    seeds = W.random_seeds(N, 121 + kind)
    g = make(native, seeds, levels=(p,))
    g.draw_u24(torch.zeros((N, 7), dtype=torch.int32, device="cuda"), 7)
    rng = np.random.Generator(np.random.PCG64(122 + kind))
    n = rng.integers(0, 5000, size=N).astype(np.uint64)
    n[:6] = [0, 1, 16, 17, 18, 2 ** 40 + 3]
    g.skip_values(torch.from_numpy(n.view(np.int64)).cuda(), kind)
    got = states(native, g, N)
    xs = seeded_X(seeds, p)
    for i in range(N):
        st = R.Stream(p, X=xs[int(seeds[i])])
        st.draw_u24(7)
        st.skip_values(int(n[i]), need)
        D, c, pos = st.D, st.c, st.pos
        assert from_limbs64(got[i, :9]) == D, i
        assert int(got[i, 9]) == c | (pos << 32), i


def test_draw_raw_lcg_doubles(native, path):
    """Raw LCG doubles (the comparison form of Sec. 2.3): per-stream counts with zeros,
    counts that end inside a refill, streams left at odd read positions by a u24 draw,
    two luxury levels; every value's bit pattern and every final state against the
    oracle's Stream.draw_raw52."""
    n = 150
    seeds = W.random_seeds(n, 91)
    levels = (223, 2048)
    level_of = (np.arange(n) % 2).astype(np.uint8)
    g = make(native, seeds, levels=levels, level_of=level_of, path=path)
    pre = (np.arange(n) * 5) % 26                        # leaves positions 0 .. 24 and 25
    po = np.concatenate([[0], np.cumsum(pre)[:-1]]).astype(np.int64)
    tmp = torch.zeros(int(pre.sum()) + 1, dtype=torch.int32, device="cuda")
    g.draw_u24(tmp, 0, torch.from_numpy(pre.astype(np.int64)).cuda(), torch.from_numpy(po).cuda())
    counts = np.array([0 if i % 13 == 0 else (i * 37) % 300 + 1 for i in range(n)], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    out = torch.full((int(counts.sum()) + 1,), -1, dtype=torch.int64, device="cuda")
    g.draw_raw_f64(out, 0, torch.from_numpy(counts).cuda(), torch.from_numpy(offs).cuda())
    got = out.cpu().numpy().view(np.uint64)
    assert got[-1] == np.uint64(2 ** 64 - 1)              # nothing past the output
    recs = states(native, g, n)
    for i in range(n):
        p = levels[int(level_of[i])]
        s = R.Stream(p, seed=int(seeds[i]))
        s.draw_u24(int(pre[i]))
        vals = s.draw_raw52(int(counts[i]))
        want = np.array([R.f64_bits(R.f64_from_bits52(v)) for v in vals], dtype=np.uint64)
        assert np.array_equal(got[offs[i]:offs[i] + counts[i]], want), i
        D, c, pos, _ = s.state()
        assert list(recs[i, :9]) == D and int(recs[i, 9]) == c | (pos << 32), i
