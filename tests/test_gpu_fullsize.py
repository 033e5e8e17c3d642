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
