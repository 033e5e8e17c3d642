"""The tensor-core refill (RLXPP_PATH_TENSOR) against the oracle and against the
integer-pipe path, bit-exact (GPU).  The exact-integer fp16 product is checked on
crafted operands, including all-ones X (the largest column sums), at several luxury
levels; the draw kernels on the tensor path must give the same values and states as
the integer path for uniform and ragged counts, odd read positions and the fused
consumer."""
import random

import numpy as np
import pytest

from oracle import ranluxpp as R
from oracle import swb_lib as S
from paper_2106_02504_gb300 import workloads as W
from tests.oracle_side import StreamSet, from_limbs64, limbs64
from tests.rare_paths import (conversion_carry_states, tc_above_m_inputs, tc_d_above_m_states,
                               tc_d_borrow_states, tc_d_limb8_carry_states, tc_limb8_carry_inputs)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def to_dev(rows):
    return torch.from_numpy(np.array(rows, dtype=np.uint64).view(np.int64)).cuda()


@pytest.mark.parametrize("p", [1, 24, 389, 2048])
def test_tc_product(native, p):
    rng = random.Random(300 + p)
    M = R.M
    A = R.luxury_multiplier(p)
    xs = [0, 1, 2, M - 1, M - 2, 2 ** 576 - 1, 2 ** 575, 2 ** 240 - 1, (2 ** 576 - 1) // 255 * 254] + \
        [rng.randrange(M) for _ in range(1000)]
    # products below 2^240 - 1 (folded to r + m: the final correction), and operands
    # whose fold carries out of limb 8 (found for the levels with dense R_j)
    xs += tc_above_m_inputs(A)
    if p in (389, 2048):
        hits = tc_limb8_carry_inputs(A, random.Random(100 + p))
        assert hits
        xs += hits
    n = len(xs)
    out = torch.zeros((n, 9), dtype=torch.int64, device="cuda")
    native.rlxpp_test_tc_mulmod(p, to_dev([limbs64(x, 9) for x in xs]), out, n)
    got = out.cpu().numpy().view(np.uint64)
    for k in range(n):
        assert from_limbs64(got[k]) == A * xs[k] % M, (p, k)


def _rare_epilogue_run(native, xs, p, per_stream):
    """From an exhausted block, every stream draws two blocks of doubles (per-stream
    counts: the kernel with operand rows holding X; one count for all: the tile-wide store
    kernel, rows holding D and c) and then the fused sum and histogram (rows holding D and
    c); values, sums and final states against the oracle."""
    n = len(xs)
    ref = StreamSet(xs, p, [24] * n)
    g = native.Generator(n, [p], torch.arange(1, n + 1, dtype=torch.int64, device="cuda"))
    g.set_path(native.RLXPP_PATH_TENSOR)
    g.set_state(ref.state_records().view(np.int64).copy())
    if per_stream:
        out = torch.zeros(n * 24, dtype=torch.float64, device="cuda")
        counts = torch.full((n,), 24, dtype=torch.int64, device="cuda")
        offsets = torch.arange(0, 24 * n, 24, dtype=torch.int64, device="cuda")
        g.draw_f64(out, 0, counts, offsets)
        out = out.view(n, 24)
    else:
        out = torch.zeros((n, 24), dtype=torch.float64, device="cuda")
        g.draw_f64(out, 24)
    want = ref.draw(24, S.KIND_F64)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want.view(np.uint64))
    assert np.array_equal(states(native, g, n).numpy().view(np.uint64), ref.state_records())
    ref = StreamSet(xs, p, [24] * n)
    g.set_state(ref.state_records().view(np.int64).copy())
    sums = torch.zeros(n, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(36, sums, hist)
    wsums, whist = ref.sum_hist(36)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64), wsums)
    assert np.array_equal(hist.cpu().numpy().view(np.uint64), whist)
    assert np.array_equal(states(native, g, n).numpy().view(np.uint64), ref.state_records())
    g.sync()
    g.close()


@pytest.mark.parametrize("p", [389, 2048])
def test_tc_draw_rare_epilogue(native, p):
    """States whose next refill takes the tensor epilogue's rare branch, each kind of
    state built for the form of operand row that meets it: for rows holding X, products
    whose fold carries past limb 8 and products below 2^240 - 1 (the final correction);
    for rows holding D and c, assembled values whose fold borrows out of limb 0 or carries
    past limb 8, and products that need the final correction; for both, products whose
    conversion carries past limb 7 or borrows past the lowest limb of its quotient
    (tests/test_rare_paths.py checks on the CPU that each reaches its case)."""
    A, M = R.luxury_multiplier(p), R.M
    Ainv = pow(A, -1, M)
    conv = [Ainv * y % M for y in conversion_carry_states(random.Random(600 + p), k=8)]
    x_form = tc_limb8_carry_inputs(A, random.Random(500 + p)) + tc_above_m_inputs(A) + conv
    d_form = (tc_d_borrow_states(A, random.Random(700 + p)) + tc_d_limb8_carry_states(A, random.Random(800 + p), want=2)
              + tc_d_above_m_states(A) + conv)
    _rare_epilogue_run(native, [x for x in x_form if 0 < x < M], p, per_stream=True)
    _rare_epilogue_run(native, [x for x in d_form if 0 < x < M], p, per_stream=False)


def pair(native, seeds, levels=(2048,)):
    d = torch.from_numpy(np.asarray(seeds, np.uint64).view(np.int64)).cuda()
    a = native.Generator(len(seeds), list(levels), d)
    a.set_path(native.RLXPP_PATH_IMAD)
    b = native.Generator(len(seeds), list(levels), d)
    b.set_path(native.RLXPP_PATH_TENSOR)
    assert native.rlxpp_get_path(a.handle) == native.RLXPP_PATH_IMAD
    assert native.rlxpp_get_path(b.handle) == native.RLXPP_PATH_TENSOR
    return a, b


def states(native, g, n):
    buf = torch.zeros((n, 11), dtype=torch.int64, device="cuda")
    g.get_state(buf)
    return buf.cpu()


def test_tc_draws_match_integer_path(native):
    n = 300
    seeds = W.random_seeds(n, 301)
    a, b = pair(native, seeds)
    ref = StreamSet.from_seeds(seeds, 2048)
    for kind, count in [(S.KIND_F64, 1000), (S.KIND_U24, 37), (S.KIND_F64, 13), (S.KIND_U24, 24)]:
        dt = torch.float64 if kind == S.KIND_F64 else torch.int32
        oa = torch.zeros((n, count), dtype=dt, device="cuda")
        ob = torch.zeros((n, count), dtype=dt, device="cuda")
        (a.draw_f64 if kind == S.KIND_F64 else a.draw_u24)(oa, count)
        (b.draw_f64 if kind == S.KIND_F64 else b.draw_u24)(ob, count)
        assert torch.equal(oa, ob), (kind, count)
        want = ref.draw(count, kind)
        got = ob.cpu().numpy()
        assert np.array_equal(got.view(np.uint64) if kind == S.KIND_F64 else got.view(np.uint32),
                              want.view(np.uint64) if kind == S.KIND_F64 else want)
    assert torch.equal(states(native, a, n), states(native, b, n))
    # ragged counts and offsets
    counts, offsets = W.ragged_counts(n, 100, seed=302)
    oa = torch.zeros(int(counts.sum()) + 1, dtype=torch.float64, device="cuda")
    ob = torch.zeros_like(oa)
    c_d, o_d = torch.from_numpy(counts).cuda(), torch.from_numpy(offsets).cuda()
    a.draw_f64(oa, 0, c_d, o_d)
    b.draw_f64(ob, 0, c_d, o_d)
    assert torch.equal(oa, ob)
    # fused consumer
    sa, sb = torch.zeros(n, dtype=torch.int64, device="cuda"), torch.zeros(n, dtype=torch.int64, device="cuda")
    ha, hb = torch.zeros(256, dtype=torch.int64, device="cuda"), torch.zeros(256, dtype=torch.int64, device="cuda")
    a.draw_f64_sum_hist(2000, sa, ha)
    b.draw_f64_sum_hist(2000, sb, hb)
    assert torch.equal(sa, sb) and torch.equal(ha, hb)
    assert torch.equal(states(native, a, n), states(native, b, n))
    b.sync()


def test_tc_path_rules(native):
    one = native.Generator(8, [2048], torch.arange(1, 9, dtype=torch.int64, device="cuda"))
    assert native.rlxpp_get_path(one.handle) == native.RLXPP_PATH_TENSOR   # single level: tensor default
    g = native.Generator(8, [24, 2048], torch.arange(1, 9, dtype=torch.int64, device="cuda"))
    assert native.rlxpp_get_path(g.handle) == native.RLXPP_PATH_TENSOR
    g.set_path(native.RLXPP_PATH_IMAD)
    with pytest.raises(native.RlxppError):
        g.set_path(7)
    assert native.rlxpp_get_path(g.handle) == native.RLXPP_PATH_IMAD


def test_tc_full_size_workload(native):
    """The 2^20-stream workload on the tensor path: sampled streams vs the oracle."""
    n = 1 << 20
    seeds = W.consecutive_seeds(n)
    g = native.Generator(n, [2048], torch.from_numpy(seeds.view(np.int64)).cuda())
    g.set_path(native.RLXPP_PATH_TENSOR)
    out = torch.empty((n, 1024), dtype=torch.float64, device="cuda")
    g.draw_f64(out, 1024)
    sums = torch.zeros(n, dtype=torch.int64, device="cuda")
    hist = torch.zeros(256, dtype=torch.int64, device="cuda")
    g.draw_f64_sum_hist(4096, sums, hist)
    g.sync()
    rng = np.random.Generator(np.random.PCG64(303))
    idx = np.unique(np.concatenate([rng.choice(n, 400, replace=False), [0, 127, 128, n - 1]]))
    ref = StreamSet.from_seeds(seeds[idx], 2048)
    want = ref.draw(1024, S.KIND_F64).view(np.uint64)
    got = out.view(torch.int64)[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint64)
    assert np.array_equal(got, want)
    wsums, _ = ref.sum_hist(4096)
    assert np.array_equal(sums.cpu().numpy().view(np.uint64)[idx], wsums)
    assert int(hist.sum()) == n * 4096


def test_bounded_wait_reports_timeout(native):
    """A wait that nothing completes gives up, reports RLXPP_ERR_TIMEOUT, and the
    context keeps working."""
    import time
    scratch = torch.zeros(9, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    with pytest.raises(native.RlxppError) as e:
        native.rlxpp_test_tc_timeout(scratch)
    assert e.value.status == native.RLXPP_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    x = torch.zeros((1, 9), dtype=torch.int64, device="cuda")
    x[0, 0] = 5
    out = torch.zeros((1, 9), dtype=torch.int64, device="cuda")
    native.rlxpp_test_tc_mulmod(2048, x, out, 1)
    assert from_limbs64(out.cpu().numpy().view(np.uint64)[0]) == R.luxury_multiplier(2048) * 5 % R.M
