"""rlxpp_seed_states_noalloc: seeding for callers that cannot allocate device memory
(an application that owns the whole memory budget, or a path where the implicit
synchronisation of cudaMalloc/cudaFree is not acceptable).  On two calls in a row that
reuse its fixed scratch array with different luxury levels it must give exactly the
records of the oracle (seed s at level p is the LCG state A_p^(2^96 s), read position
0) and of the allocating path (rlxpp_create followed by rlxpp_get_state), and it must
allocate nothing: with the library's allocation countdown set to fail the very next
allocation it still succeeds, and the device's free memory does not change.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

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


def _records_allocating_path(native, levels, seeds_d, level_of_d, n):
    g = native.Generator(n, levels, seeds_d, level_of_d)
    ref = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    g.get_state(ref)
    g.sync()
    g.close()
    return ref


def _records_oracle(levels, seeds, level_of):
    """(n, 11) uint64 records from the oracle, stream by stream at its own level."""
    n = len(seeds)
    lv = np.zeros(n, dtype=np.int64) if level_of is None else level_of.astype(np.int64)
    rec = np.zeros((n, 11), dtype=np.uint64)
    for li, p in enumerate(levels):
        sel = np.nonzero(lv == li)[0]
        if sel.size:
            rec[sel] = StreamSet.from_seeds(seeds[sel], p).state_records()
    return rec


def _calls(n):
    return [([2048], 11, None),
            ([24, 223, 389, 2048], 12, W.batch_mix(n, seed=13)[1])]


def test_noalloc_seeding_matches_oracle_and_allocating_path(native):
    n = 1000  # several 128-thread blocks and a ragged tail
    for levels, seed, level_of in _calls(n):   # two calls in a row share the scratch array
        seeds = W.random_seeds(n, seed)
        seeds[:3] = [1, 2, 2 ** 64 - 1]
        seeds_d = torch.from_numpy(seeds.view(np.int64)).cuda()
        level_of_d = None if level_of is None else torch.from_numpy(level_of).cuda()
        out = torch.full((n, 11), -1, dtype=torch.int64, device="cuda")
        native.rlxpp_seed_states_noalloc(levels, seeds_d, n, out, level_of_d)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, _records_oracle(levels, seeds, level_of)), levels
        ref = _records_allocating_path(native, levels, seeds_d, level_of_d, n)
        assert torch.equal(out, ref), levels


def test_noalloc_allocates_nothing(native):
    """With every input and output already on the device, two calls in a row succeed
    while the library's next device allocation is set to fail, and the device's free
    memory is the same before and after them."""
    n = 700
    prepared = []
    for levels, seed, level_of in _calls(n):
        seeds = W.random_seeds(n, seed + 100)
        prepared.append((levels, seeds, torch.from_numpy(seeds.view(np.int64)).cuda(),
                         None if level_of is None else torch.from_numpy(level_of).cuda(), level_of))
    outs = [torch.full((n, 11), -1, dtype=torch.int64, device="cuda") for _ in prepared]
    levels0, _, seeds0, lvl0, _ = prepared[0]
    native.rlxpp_seed_states_noalloc(levels0, seeds0, n, outs[0], lvl0)   # the device's first call
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    native.rlxpp_test_fail_alloc(0)       # the library's next device allocation fails
    try:
        for (levels, _, seeds_d, level_of_d, _), out in zip(prepared, outs):
            native.rlxpp_seed_states_noalloc(levels, seeds_d, n, out, level_of_d)
        torch.cuda.synchronize()
    finally:
        native.rlxpp_test_fail_alloc(-1)
    assert torch.cuda.mem_get_info()[0] == free0
    for (levels, seeds, _, _, level_of), out in zip(prepared, outs):
        assert np.array_equal(out.cpu().numpy().view(np.uint64), _records_oracle(levels, seeds, level_of)), levels


def test_noalloc_limits(native):
    seeds = torch.ones(4, dtype=torch.int64, device="cuda")
    out = torch.zeros((4, 11), dtype=torch.int64, device="cuda")
    with pytest.raises(native.RlxppError) as e:
        native.rlxpp_seed_states_noalloc([24, 48, 97, 223, 389], seeds, 4, out)   # 5 > 4 levels
    assert e.value.status == native.RLXPP_ERR_INVALID
    with pytest.raises(native.RlxppError):
        native.rlxpp_seed_states_noalloc([2048], seeds.cpu(), 4, out)             # host seeds
    # a level index beyond the list, or a zero seed, gives an all-zero (invalid, p = 0)
    # record
    lvl = torch.tensor([0, 1, 0, 0], dtype=torch.uint8, device="cuda")
    seeds[3] = 0
    native.rlxpp_seed_states_noalloc([2048], seeds, 4, out, lvl)
    torch.cuda.synchronize()
    assert int(out[1].abs().sum()) == 0 and int(out[3].abs().sum()) == 0 and int(out[0, 10]) == 2048
