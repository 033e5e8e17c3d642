"""Asynchronous draws into page-locked host memory (GPU): the values equal the oracle's
(sampled streams, the staging chunks' edges included), a device draw queued behind one
on the same stream continues each stream's sequence without waiting for the copies, the
staging buffer is reused and grown across calls, and pageable or device outputs are
rejected."""
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


@pytest.mark.parametrize("path", ["tensor", "imad"])
def test_async_host_draws(native, path):
    n, cnt = 70_000, 1024                       # 573 MB: three 256 MB staging chunks
    chunk = (256 << 20) // (cnt * 8)
    seeds = np.arange(1, n + 1, dtype=np.uint64)
    g = native.Generator(n, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_TENSOR if path == "tensor" else native.RLXPP_PATH_IMAD)
    rng = np.random.Generator(np.random.PCG64(43))
    edges = {0, 1, chunk - 1, chunk, 2 * chunk - 1, 2 * chunk, n - 1}
    idx = np.array(sorted(set(rng.choice(n, 120, replace=False).tolist()) | edges))
    ref = StreamSet.from_seeds(seeds[idx], 2048)

    host = torch.empty((n, cnt), dtype=torch.float64).pin_memory()
    nxt = torch.empty((n, 10), dtype=torch.float64, device="cuda")
    g.draw_f64_host_async(host, cnt)
    g.draw_f64(nxt, 10)                          # same stream, behind the compute only
    g.host_wait()
    torch.cuda.current_stream().synchronize()
    got = host.numpy().view(np.uint64)[idx]
    assert np.array_equal(got, ref.draw(cnt, S.KIND_F64).view(np.uint64))
    got = nxt.cpu().numpy().view(np.uint64)[idx]
    assert np.array_equal(got, ref.draw(10, S.KIND_F64).view(np.uint64))

    # the staging buffer reused (smaller) and then grown (larger), u24 and f64
    small = torch.empty((n, 100), dtype=torch.int32).pin_memory()
    g.draw_u24_host_async(small, 100)
    big = torch.empty((n, 1500), dtype=torch.float64).pin_memory()
    g.draw_f64_host_async(big, 1500)
    g.host_wait()
    torch.cuda.current_stream().synchronize()
    assert np.array_equal(small.numpy().view(np.uint32)[idx], ref.draw(100, S.KIND_U24))
    assert np.array_equal(big.numpy().view(np.uint64)[idx], ref.draw(1500, S.KIND_F64).view(np.uint64))

    # outputs that are not page-locked host memory are rejected, the streams untouched
    for bad in (torch.empty((n, 5), dtype=torch.float64), torch.empty((n, 5), dtype=torch.float64, device="cuda")):
        with pytest.raises(native.RlxppError) as err:
            g.draw_f64_host_async(bad, 5)
        assert err.value.status == native.RLXPP_ERR_INVALID
    g.draw_f64(nxt, 10)
    torch.cuda.synchronize()
    assert np.array_equal(nxt.cpu().numpy().view(np.uint64)[idx], ref.draw(10, S.KIND_F64).view(np.uint64))
    g.close()


def test_async_host_draw_edge_cases(native):
    """Zero counts and an empty generator return at once without touching the output;
    waiting with nothing in flight is a no-op; the streams do not move."""
    g = native.Generator(5, [2048], torch.arange(1, 6, dtype=torch.int64, device="cuda"))
    ref = StreamSet.from_seeds(np.arange(1, 6, dtype=np.uint64), 2048)
    g.host_wait()                                     # nothing issued yet
    host = torch.full((5, 3), 7.0, dtype=torch.float64).pin_memory()
    g.draw_f64_host_async(host, 0)
    g.host_wait()
    torch.cuda.synchronize()
    assert bool((host == 7.0).all())
    out = torch.empty((5, 4), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 4)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint64), ref.draw(4, S.KIND_F64).view(np.uint64))
    g.close()
    e = native.Generator(0, [2048], None)
    e.draw_u24_host_async(torch.empty((0, 8), dtype=torch.int32).pin_memory(), 8)
    e.host_wait()
    torch.cuda.synchronize()
    e.close()
