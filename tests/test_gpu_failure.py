"""Failure paths on the host side (GPU present, nothing faults): device allocations made
to fail by the library's test countdown (rlxpp_test_fail_alloc) at every allocation
point of rlxpp_create and of a draw into host memory.  Each failing call must return
RLXPP_ERR_NOMEM, release what it had allocated, and leave an existing generator's
streams where they were; the next call must work and give the oracle's values."""
import numpy as np
import pytest

from oracle import swb_lib as S
from tests.oracle_side import StreamSet

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


@pytest.fixture(autouse=True)
def countdown_off(native):
    yield
    native.rlxpp_test_fail_alloc(-1)


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_create_fails_cleanly_at_every_allocation(native):
    n = 200_000                                    # 14 MB of state: a leak would show
    seeds = np.arange(1, n + 1, dtype=np.uint64)
    native.rlxpp_destroy(native.rlxpp_create(n, [2048, 24], seeds))   # context and pools warm
    before = free_bytes()
    outcomes = []
    for after in range(40):
        native.rlxpp_test_fail_alloc(after)
        try:
            h = native.rlxpp_create(n, [2048, 24], seeds)
        except native.RlxppError as e:
            assert e.status == native.RLXPP_ERR_NOMEM, str(e)
            outcomes.append("nomem")
        else:
            native.rlxpp_destroy(h)
            outcomes.append("ok")
        native.rlxpp_test_fail_alloc(-1)
        if outcomes[-1] == "ok":
            break
    # every allocation point before the last one failed the call; then it succeeds
    assert outcomes[-1] == "ok" and outcomes.count("nomem") == len(outcomes) - 1 >= 7
    assert abs(free_bytes() - before) <= 4 << 20          # nothing left allocated
    # and a generator created afterwards is correct
    m = 5000
    g = native.Generator(m, [2048], torch.from_numpy(seeds[:m].view(np.int64)).cuda())
    out = torch.zeros((m, 30), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 30)
    want = StreamSet.from_seeds(seeds[:m], 2048).draw(30, S.KIND_F64)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want.view(np.uint64))
    g.close()


@pytest.mark.parametrize("path", ["tensor", "imad"])
def test_draw_to_host_fails_cleanly(native, path):
    # 140,000 streams x 250 doubles = 280 MB of host output: two 256 MB staging chunks
    n, cnt = 140_000, 250
    chunk = (256 << 20) // (cnt * 8)
    seeds = np.arange(1, n + 1, dtype=np.uint64)
    g = native.Generator(n, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_TENSOR if path == "tensor" else native.RLXPP_PATH_IMAD)
    rng = np.random.Generator(np.random.PCG64(41))
    idx = np.array(sorted(set(rng.choice(n, 150, replace=False).tolist()) | {0, 1, chunk - 1, chunk, n - 1}))
    ref = StreamSet.from_seeds(seeds[idx], 2048)
    host = torch.zeros((n, cnt), dtype=torch.float64)

    def check(t, k):
        got = t.numpy().view(np.uint64).reshape(n, k)[idx]
        assert np.array_equal(got, ref.draw(k, S.KIND_F64).view(np.uint64))

    # the first staging buffer fails: nothing is drawn, the streams stay put
    native.rlxpp_test_fail_alloc(0)
    with pytest.raises(native.RlxppError) as err:
        g.draw_f64(host, cnt)
    assert err.value.status == native.RLXPP_ERR_NOMEM
    native.rlxpp_test_fail_alloc(-1)
    assert not bool(host.any())
    g.draw_f64(host, cnt)
    check(host, cnt)
    # the second staging buffer fails: both chunks go through the one buffer
    native.rlxpp_test_fail_alloc(1)
    g.draw_f64(host, cnt)
    native.rlxpp_test_fail_alloc(-1)
    check(host, cnt)
    # per-stream counts into host memory: its one staging buffer fails
    counts = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    offsets = torch.arange(n, dtype=torch.int64, device="cuda") * 7
    flat = torch.zeros(7 * n, dtype=torch.float64)
    native.rlxpp_test_fail_alloc(0)
    with pytest.raises(native.RlxppError) as err:
        g.draw_f64(flat, 0, counts, offsets)
    assert err.value.status == native.RLXPP_ERR_NOMEM
    native.rlxpp_test_fail_alloc(-1)
    g.draw_f64(flat, 0, counts, offsets)
    check(flat, 7)
    g.close()
