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


def test_cursor_arithmetic_matches_oracle_rule():
    from paper_2106_02504_gb300.serve import advance_cursor
    from oracle import ranluxpp as R
    st = R.Stream(24, seed=3)
    block, pos = 0, 0
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(200):
        kind, count = int(rng.integers(0, 2)), int(rng.integers(0, 40))
        (st.draw_f64 if kind == 1 else st.draw_u24)(count)
        block, pos = advance_cursor(block, pos, kind, count)
        assert pos == st.pos
        # the stream's LCG state sits `block` advances after the seeded state
        assert pow(R.luxury_multiplier(24), block, R.M) * R.seed_lcg(3, 24) % R.M == st.X


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
