"""The 2^20-stream workload at full size on the integer-pipe path (the tensor path has its
own full-size test), in the launch configuration bench.py times
(rlxpp_seed, rlxpp_draw_f64 of 1024 doubles per stream into an 8 GiB device buffer,
rlxpp_draw_f64_sum_hist of 4096 doubles per stream), checked bit-exactly against the
oracle on sampled streams (every output of each sampled stream, and its final state)
and through properties that hold at any size (histogram total, range and bit pattern
of every double)."""
import numpy as np
import pytest

from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import StreamSet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 1 << 20
P = 2048


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P_
    return P_.native


def sample_idx(seed, k=1500):
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = set(rng.choice(N, size=k, replace=False).tolist())
    idx |= {0, 1, 31, 32, 127, 128, 4095, N // 2, N - 2, N - 1}
    return np.array(sorted(idx))


def test_hbm_workload_full_size(native):
    seeds = W.consecutive_seeds(N)
    g = native.Generator(N, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_IMAD)
    g.seed(torch.from_numpy(seeds.view(np.int64)).cuda())
    out = torch.empty((N, 1024), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 1024)
    torch.cuda.synchronize()
    bits = out.view(torch.int64)
    # every double in [0, 1) with at most 48 significant bits below its leading one
    assert int(bits.min()) >= 0 and int(bits.max()) < 0x3FF0000000000000
    nz = bits[bits != 0]
    mant = (nz & ((1 << 52) - 1)) | (1 << 52)
    assert int((mant & 0x1F).max()) == 0   # v 2^-48 with v < 2^48: 5 trailing zero bits at least
    # distinct streams: first values pairwise different on a sample
    idx = sample_idx(1)
    ref = StreamSet.from_seeds(seeds[idx], P)
    want = ref.draw(1024, S.KIND_F64).view(np.uint64)
    got = bits[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"streams {idx[bad[:5]]} differ"
    st = torch.zeros((N, 11), dtype=torch.int64, device="cuda")
    g.get_state(st)
    gs = st[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    assert np.array_equal(gs, ref.state_records())
    del out, bits
    g.close()


def test_fused_workload_full_size(native):
    seeds = W.consecutive_seeds(N)
    g = native.Generator(N, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_IMAD)
    sums = torch.zeros(N, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(4096, sums, hist)
    torch.cuda.synchronize()
    assert int(hist.sum()) == N * 4096
    idx = sample_idx(2, k=600)
    ref = StreamSet.from_seeds(seeds[idx], P)
    wsums, whist = ref.sum_hist(4096)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64)[idx], wsums)
    # the sampled streams' histogram is bounded by the full histogram bin by bin
    assert (hist.cpu().numpy().view(np.uint64) >= whist).all()
    g.close()


@pytest.mark.parametrize("path", ["tensor", "imad"])
def test_output_past_2_32_elements(native, path):
    """More than 2^32 output elements in one call (2^20 streams x 4100 u24 = 4.3e9
    values, 17.2 GB): element offsets, tile coordinates and the tensor map's extents
    pass 32 bits; sampled streams, the last ones included, equal the oracle."""
    n, cnt = N, 4100
    assert n * cnt > 2 ** 32
    seeds = W.consecutive_seeds(n)
    g = native.Generator(n, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_IMAD if path == "imad" else native.RLXPP_PATH_TENSOR)
    out = torch.empty((n, cnt), dtype=torch.int32, device="cuda")
    g.draw_u24(out, cnt)
    torch.cuda.synchronize()
    idx = np.array(sorted(set(sample_idx(3, k=200).tolist()) | {n - 129, n - 128, n - 3}))
    ref = StreamSet.from_seeds(seeds[idx], P)
    want = ref.draw(cnt, S.KIND_U24)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint32)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"streams {idx[bad[:5]]} differ"
    # every value is a 24-bit number
    assert int(out.max()) < 2 ** 24 and int(out.min()) >= 0
    del out
    g.close()


def test_config1_single_stream_serial_full_size(native):
    """One stream (seed 1, p = 2048) read in order on the path bench.py times for it (one
    warp per stream): 2^20 doubles, and separately 2^20 u24 from a fresh seed-1 state,
    every value against the oracle."""
    n = 1 << 20
    for kind in (S.KIND_F64, S.KIND_U24):
        g = native.Generator(1, [P], torch.ones(1, dtype=torch.int64, device="cuda"))
        g.set_path(native.RLXPP_PATH_WARP)
        dt = torch.float64 if kind == S.KIND_F64 else torch.int32
        out = torch.empty(n, dtype=dt, device="cuda")
        (g.draw_f64 if kind == S.KIND_F64 else g.draw_u24)(out, n)
        torch.cuda.synchronize()
        ref = StreamSet.from_seeds([1], P)
        want = ref.draw(n, kind)[0]
        got = out.cpu().numpy()
        if kind == S.KIND_F64:
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64))
        else:
            assert np.array_equal(got.view(np.uint32), want)
        st = torch.zeros((1, 11), dtype=torch.int64, device="cuda")
        g.get_state(st)
        assert np.array_equal(st.cpu().numpy().view(np.uint64), ref.state_records())
        g.close()


def test_config3_mixed_batch_full_size(native):
    """The mixed batch at full size (65,536 streams, levels {24, 223, 389, 2048}, counts
    log-uniform in [1, 10^6], u24/f64 50/50, seeds i + 1) as one planned run on the tensor
    request kernel: sampled requests, the longest included, equal the oracle value by
    value; the output totals and the untouched tail are checked whole."""
    import paper_2106_02504_gb300._rlxpp as B
    n = 65536
    levels, lvl, counts, is_f64 = W.batch_mix(n, seed=3)
    seeds = np.arange(1, n + 1, dtype=np.uint64)
    g = native.Generator(n, levels, torch.from_numpy(seeds.view(np.int64)).cuda(), torch.from_numpy(lvl).cuda())
    reqs = np.zeros(n, dtype=B.request_dtype())
    reqs["stream"] = np.arange(n)
    reqs["kind"] = is_f64.astype(np.uint32)
    reqs["count"] = counts
    off = np.zeros(n, dtype=np.int64)
    for k in (0, 1):
        sel = is_f64 == bool(k)
        off[sel] = np.concatenate([[0], np.cumsum(counts[sel])[:-1]])
    reqs["offset"] = off
    nf, nu = int(counts[is_f64].sum()), int(counts[~is_f64].sum())
    out_f = torch.full((nf + 1,), -1, dtype=torch.int64, device="cuda")
    out_u = torch.full((nu + 1,), -1, dtype=torch.int32, device="cuda")
    plan = native.rlxpp_plan_requests(g.handle, reqs, 0, (128, 4, native.RLXPP_PATH_TENSOR))
    native.rlxpp_run_plan(g.handle, plan, out_u, out_f)
    torch.cuda.synchronize()
    native.rlxpp_destroy_plan(plan)
    assert int(out_f[-1]) == -1 and int(out_u[-1]) == -1            # nothing past the outputs
    assert int((out_u[:-1] < 0).sum()) == 0 and int((out_u[:-1] >= 2 ** 24).sum()) == 0
    rng = np.random.Generator(np.random.PCG64(17))
    sample = set(rng.choice(n, size=40, replace=False).tolist()) | set(np.argsort(counts)[-4:].tolist())
    for i in sorted(sample):
        ref = StreamSet.from_seeds([int(seeds[i])], levels[int(lvl[i])])
        c, o = int(counts[i]), int(off[i])
        if is_f64[i]:
            want = ref.draw(c, S.KIND_F64)[0].view(np.uint64)
            got = out_f[o:o + c].cpu().numpy().view(np.uint64)
        else:
            want = ref.draw(c, S.KIND_U24)[0]
            got = out_u[o:o + c].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want), (i, c)
    g.close()


def test_config4_skips_full_size(native):
    """2^18 streams (seeds i + 1, p = 2048) skipped by uniform 128-bit distances, then 48
    doubles each, as bench.py times it: sampled streams against pow(A, n, m)."""
    from oracle import ranluxpp as R
    from tests.oracle_side import seeded_X
    n = 1 << 18
    seeds = W.consecutive_seeds(n)
    g = native.Generator(n, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    dist = W.skip_distances(n, seed=4)
    g.skip(torch.from_numpy(dist.view(np.int64)).cuda())
    out = torch.empty((n, 48), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 48)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(18))
    idx = np.array(sorted(set(rng.choice(n, size=300, replace=False).tolist()) | {0, n - 1}))
    A = R.luxury_multiplier(P)
    xs = seeded_X(seeds[idx], P)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    for r, i in enumerate(idx):
        d = int(dist[i, 0]) | (int(dist[i, 1]) << 64)
        X = pow(A, d, R.M) * xs[int(seeds[i])] % R.M
        want = StreamSet([X], P).draw(48, S.KIND_F64)[0].view(np.uint64)
        assert np.array_equal(got[r], want), i
    g.close()


@pytest.mark.parametrize("kind", ["normal", "exponential"])
def test_distributions_full_size(native, kind):
    """Gaussian and exponential doubles as bench.py times them: 2^20 streams (seeds
    1..2^20, p = 2048) x 1024 values on the tensor path into an 8 GiB buffer; sampled
    streams against the oracle within the derived tolerances, and properties of every
    value (finite; exponential values non-negative and at most 48 ln 2; Gaussian values
    at most sqrt(96 ln 2) in magnitude, and sample moments near 0 and 1)."""
    from tests.oracle_side import exponentials_expected, normals_expected
    seeds = W.consecutive_seeds(N)
    g = native.Generator(N, [P], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_TENSOR)
    out = torch.empty((N, 1024), dtype=torch.float64, device="cuda")
    (g.draw_normal_f64 if kind == "normal" else g.draw_exp_f64)(out, 1024)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    if kind == "normal":
        assert float(out.abs().max()) <= np.sqrt(96 * np.log(2))
        m, v = float(out.mean()), float(out.var())
        assert abs(m) < 1e-3 and abs(v - 1) < 1e-3
    else:
        assert float(out.min()) >= 0 and float(out.max()) <= 48 * np.log(2)
        assert abs(float(out.mean()) - 1) < 1e-3
    idx = sample_idx(5, k=400)
    got = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = StreamSet.from_seeds(seeds[idx], P)
    d = ref.draw(1024, S.KIND_F64)
    want, tol = normals_expected(d, 1024) if kind == "normal" else exponentials_expected(d)
    bad = np.nonzero((np.abs(got - want) > tol).any(axis=1))[0]
    assert bad.size == 0, f"streams {idx[bad[:5]]} differ"
    del out
    g.close()
