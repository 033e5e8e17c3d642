"""Device arithmetic against the oracle, element by element, bit-exact (GPU).

multiply9x9 (Sec. 2.1), mod_m (Sec. 2.2), the conversions of Sec. 2.3, the double
construction and the luxury multiplier, each on crafted edge cases and seeded random
inputs, through the C-ABI test entry points."""
import random

import numpy as np
import pytest

from oracle import ranluxpp as R
from tests.oracle_side import MASK64, conversion_edge_states, from_limbs64, limbs64
from tests.rare_paths import conversion_carry_states, mod_m_carry_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def to_dev(rows):
    a = np.array(rows, dtype=np.uint64)
    return torch.from_numpy(a.view(np.int64)).cuda()


def from_dev(t):
    return t.cpu().numpy().view(np.uint64)


M = R.M
EDGE_X = [0, 1, 2, 3, M - 1, M - 2, 2 ** 575, 2 ** 576 - 2 ** 240, 2 ** 336, 2 ** 336 - 1,
          2 ** 240, 2 ** 240 - 1, 2 ** 240 - 2, M - 2 ** 240, (M - 1) // 2, 2 ** 32 - 1, 2 ** 64]


def test_luxury_multiplier(native):
    for p in (1, 2, 3, 23, 24, 25, 223, 389, 2048, 65537, 2 ** 31 + 5, 2 ** 32 - 1):
        assert native.rlxpp_luxury_multiplier(p) == R.luxury_multiplier(p), p


def test_multiply9x9(native):
    rng = random.Random(21)
    xs = [0, 1, 2 ** 576 - 1, M - 1, 2 ** 575] + [rng.randrange(2 ** 576) for _ in range(3000)]
    ys = [2 ** 576 - 1, 2 ** 576 - 1, 2 ** 576 - 1, M - 1, 2 ** 575] + \
         [rng.randrange(2 ** 576) for _ in range(3000)]
    n = len(xs)
    x, y = to_dev([limbs64(v, 9) for v in xs]), to_dev([limbs64(v, 9) for v in ys])
    out = torch.zeros((n, 18), dtype=torch.int64, device="cuda")
    native.rlxpp_test_multiply9x9(x, y, out, n)
    got = from_dev(out)
    for k in range(n):
        assert from_limbs64(got[k]) == R.multiply9x9(xs[k], ys[k]), k


def _mod_m_inputs():
    rng = random.Random(22)
    v = [0, 1, M - 1, M, M + 1, 2 * M - 1, 2 * M, 2 ** 576 - 1, 2 ** 576, (M - 1) ** 2,
         2 ** 1152 - 1, 3 * M, 4 * M + 5, 2 ** 577 - 1, 2 ** 816, 2 ** 816 - 1, 2 ** 912 - 1]
    # values whose reduction lands in [m, 2^576): m + r with r < 2^240 - 1, as products
    v += [M + r for r in (0, 1, 2 ** 239, 2 ** 240 - 2)]
    v += [k * M + r for k in (1, 2, 2 ** 100, 2 ** 575) for r in (0, 1, M - 1, 2 ** 240 - 2)]
    # high halves with special structure (H0, H1 all ones / zero)
    for H in (0, 1, 2 ** 336 - 1, 2 ** 576 - 1, 2 ** 576 - 2 ** 336, (2 ** 240 - 1) << 336):
        for L in (0, 1, 2 ** 576 - 1, M - 1, M):
            v.append((H << 576) + L if L < 2 ** 576 else (H << 576) + (L % 2 ** 576))
    v += [rng.randrange(2 ** 1152) for _ in range(4000)]
    v += [rng.randrange(M) * rng.randrange(M) for _ in range(4000)]
    # carries past limbs 7, 8 and 17 in the reduction's chains (rare for random inputs)
    v += mod_m_carry_inputs(random.Random(26))
    return [x for x in v if 0 <= x < 2 ** 1152]


@pytest.mark.parametrize("form", ["thread", "warp"])
def test_mod_m(native, form):
    """mod_m on crafted inputs (values near m and 2m, reductions that land in [m, 2^576),
    special high halves) and random ones, in the per-thread and the warp-cooperative form."""
    vals = _mod_m_inputs()
    n = len(vals)
    inp = to_dev([limbs64(v, 18) for v in vals])
    out = torch.zeros((n, 9), dtype=torch.int64, device="cuda")
    (native.rlxpp_test_mod_m if form == "thread" else native.rlxpp_test_warp_mod_m)(inp, out, n)
    got = from_dev(out)
    for k in range(n):
        assert from_limbs64(got[k]) == R.mod_m(vals[k]), hex(vals[k])


def test_mul_mod(native):
    rng = random.Random(23)
    xs = EDGE_X + [rng.randrange(M) for _ in range(3000)]
    ys = list(reversed(EDGE_X)) + [rng.randrange(M) for _ in range(3000)]
    n = len(xs)
    out = torch.zeros((n, 9), dtype=torch.int64, device="cuda")
    native.rlxpp_test_mul_mod(to_dev([limbs64(v, 9) for v in xs]), to_dev([limbs64(v, 9) for v in ys]),
                              out, n)
    got = from_dev(out)
    for k in range(n):
        assert from_limbs64(got[k]) == xs[k] * ys[k] % M, k


@pytest.mark.parametrize("form", ["thread", "warp"])
def test_conversions(native, form):
    """The conversion to RANLUX numbers (and back) on edge and random states, the
    corners where the quotient's borrow cannot be decided from the top limbs included,
    in the per-thread and the warp-cooperative form."""
    rng = random.Random(24)
    xs = [x for x in EDGE_X if 0 < x < M] + [rng.randrange(1, M) for _ in range(5000)]
    xs += conversion_edge_states(rng)
    xs += conversion_carry_states(random.Random(27))  # X + q carries past limbs 7 and 8
    n = len(xs)
    d = torch.zeros((n, 9), dtype=torch.int64, device="cuda")
    carry = torch.zeros(n, dtype=torch.int32, device="cuda")
    (native.rlxpp_test_to_ranlux if form == "thread" else native.rlxpp_test_warp_to_ranlux)(
        to_dev([limbs64(v, 9) for v in xs]), d, carry, n)
    gd, gc = from_dev(d), carry.cpu().numpy()
    for k in range(n):
        D, c = R.to_ranlux(xs[k])
        assert from_limbs64(gd[k]) == D and int(gc[k]) == c, k
    back = torch.zeros((n, 9), dtype=torch.int64, device="cuda")
    native.rlxpp_test_to_lcg(d, carry, back, n)
    gb = from_dev(back)
    for k in range(n):
        assert from_limbs64(gb[k]) == xs[k], k


def test_f64_from48(native):
    rng = np.random.Generator(np.random.PCG64(25))
    v = np.concatenate([np.array([0, 1, 2, 3, 2 ** 47, 2 ** 47 - 1, 2 ** 48 - 1, 2 ** 40, 2 ** 24 - 1],
                                 dtype=np.uint64),
                        np.array([1 << k for k in range(48)], dtype=np.uint64),
                        rng.integers(0, 2 ** 48, size=100_000, dtype=np.uint64)])
    n = len(v)
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    native.rlxpp_test_f64_from48(torch.from_numpy(v.view(np.int64)).cuda(), out, n)
    got = out.cpu().numpy().view(np.uint64)
    want = (v.astype(np.float64) * 2.0 ** -48).view(np.uint64)   # exact: v < 2^53
    assert np.array_equal(got, want)
    for x in (0, 1, 2 ** 48 - 1):
        assert int(got[list(v).index(x)]) == R.f64_bits(R.f64_from_bits48(x))


def test_empty_inputs(native):
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    native.rlxpp_test_mod_m(out, out, 0)
    native.rlxpp_test_f64_from48(out, out, 0)
    torch.cuda.synchronize()
