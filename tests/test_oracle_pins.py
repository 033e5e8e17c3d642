"""Pins of the CPU oracle to what the paper and the mathematics fix (no GPU needed).

Each test checks the oracle against something other than itself: the subtract-with-
borrow recurrence run step by step (the definition of RANLUX), closed forms derived by
hand, algebraic invariants, and values the paper prints.  A plausible mistake in the
oracle (a wrong lag, a dropped borrow, a wrong shift in the conversion, a wrong
exponent in seeding, a transposed word pair in the 48-bit draw) fails one of them.
"""
import os
import random

import numpy as np
import pytest

from oracle import ranluxpp as R
from oracle import swb_lib as S
from tests.oracle_side import conversion_edge_states

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_constants():
    out = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = (t.strip() for t in line.split("="))
                out[k] = v
    return out


def _random_swb_state(rng, warmup=48):
    """A state reached by running the recurrence (canonical for the LCG map)."""
    w = [rng.randrange(R.BASE) for _ in range(24)]
    c = rng.randrange(2)
    return R.swb_steps(w, c, warmup)


# --- constants the paper prints ---------------------------------------------------
def test_modulus_is_the_papers():
    pc = _paper_constants()
    assert pc["modulus_formula"] == "2^576 - 2^240 + 1"
    assert R.M == 2 ** 576 - 2 ** 240 + 1           # Sec. 2.2
    assert R.M == R.BASE ** 24 - R.BASE ** 10 + 1   # b^r - b^s + 1
    assert R.STATE_BITS == int(pc["state_bits"]) == 64 * int(pc["state_limbs_u64"])
    assert int(pc["double_bits"]) == 48
    assert R.SEED_SHIFT == int(pc["seed_skip_exponent"])


def test_one_step_multiplier_closed_form():
    # a = m - (m - 1) / 2^24, (m - 1) / 2^24 = 2^552 - 2^216, derived by hand.
    a = R.one_step_multiplier()
    assert a == 2 ** 576 - 2 ** 552 - 2 ** 240 + 2 ** 216 + 1
    assert (a * R.BASE - 1) % R.M == 0
    # sparse form a = 2^216 - 2^552 (mod m)
    assert (a - (2 ** 216 - 2 ** 552)) % R.M == 0


def test_luxury_multiplier_small_powers():
    a = R.one_step_multiplier()
    assert R.luxury_multiplier(1) == a
    assert R.luxury_multiplier(2) == a * a % R.M
    assert R.luxury_multiplier(0) == 1
    # a^24 = b^-24 = 2^-576 = (2^240 - 1)^-1 mod m
    assert R.luxury_multiplier(24) * (2 ** 240 - 1) % R.M == 1


# --- the LCG equals the recurrence --------------------------------------------------
def test_lcg_equals_swb_p24_ten_thousand():
    """10,000 single LCG advances at p = 24, each against 24 recurrence steps."""
    p = 24
    A = R.luxury_multiplier(p)
    w, c = R.to_ranlux(R.seed_lcg(1, p))
    w = R.unpack_words(w)
    X = R.to_lcg(R.pack_words(w), c)
    for _ in range(10_000):
        w, c = R.swb_steps(w, c, p)
        X = R.advance(X, A)
        D, cx = R.to_ranlux(X)
        assert R.unpack_words(D) == w and cx == c
        assert R.to_lcg(R.pack_words(w), c) == X


@pytest.mark.parametrize("p", [1, 2, 7, 23, 24, 25, 223, 389, 2048])
def test_lcg_equals_swb_various_p(p):
    rng = random.Random(1000 + p)
    A = R.luxury_multiplier(p)
    for _ in range(20):
        w, c = _random_swb_state(rng)
        X = R.to_lcg(R.pack_words(w), c)
        w2, c2 = S.block(w, c, p)           # C recurrence
        if p <= 400:
            assert (w2, c2) == tuple(R.swb_steps(w, c, p))  # Python recurrence
        D, cx = R.to_ranlux(R.advance(X, A))
        assert R.unpack_words(D) == w2 and cx == c2


def test_c_and_python_recurrence_agree():
    rng = random.Random(7)
    for _ in range(50):
        w = [rng.randrange(R.BASE) for _ in range(24)]
        c = rng.randrange(2)
        n = rng.randrange(1, 100)
        assert S.block(w, c, n) == tuple(R.swb_steps(w, c, n))


def test_recurrence_hand_values():
    """One step on hand-made windows: x_n = x_{n-10} - x_{n-24} - c mod 2^24."""
    w = list(range(24))            # w[0] = 0 is x_{n-24}, w[14] = 14 is x_{n-10}
    w2, c2 = R.swb_step(w, 0)
    assert w2[-1] == 14 and c2 == 0 and w2[:-1] == w[1:]
    w = [5] + [0] * 23             # 0 - 5 - 1 = -6 -> 2^24 - 6, borrow 1
    w2, c2 = R.swb_step(w, 1)
    assert w2[-1] == 2 ** 24 - 6 and c2 == 1
    assert S.block([5] + [0] * 23, 1, 1) == ([0] * 23 + [2 ** 24 - 6], 1)


# --- conversions ----------------------------------------------------------------------
def test_conversion_round_trip_and_range():
    rng = random.Random(3)
    xs = [1, 2, 3, R.M - 1, R.M - 2, 2 ** 575, 2 ** 576 - 2 ** 240, 2 ** 336, 2 ** 336 - 1,
          2 ** 240, 2 ** 240 - 1] + [rng.randrange(1, R.M) for _ in range(2000)]
    edges = conversion_edge_states(rng)
    xs += edges
    for X in xs:
        D, c = R.to_ranlux(X)
        assert c in (0, 1)
        assert 0 <= D < 2 ** 576
        assert R.to_lcg(D, c) == X
        # D / 2^576 approximates X / m from below within 2^-576
        assert D * R.M <= X * 2 ** 576 < (D + 1) * R.M
    # the corner states include quotients by m one above the quotient by 2^576
    over = [X for X in edges if R.to_ranlux(X)[0] != X + (X * (2 ** 240 - 1) >> 576)]
    assert len(over) >= 7


def test_conversion_inverts_recurrence_states():
    rng = random.Random(5)
    for _ in range(500):
        w, c = _random_swb_state(rng)
        X = R.to_lcg(R.pack_words(w), c)
        assert 0 < X < R.M
        D, c2 = R.to_ranlux(X)
        assert R.unpack_words(D) == w and c2 == c


# --- modulo ---------------------------------------------------------------------------
def test_mod_m_closed_forms():
    M = R.M
    assert R.mod_m(0) == 0
    assert R.mod_m(1) == 1
    assert R.mod_m(M - 1) == M - 1
    assert R.mod_m(M) == 0
    assert R.mod_m(M + 1) == 1
    assert R.mod_m(2 * M - 1) == M - 1
    assert R.mod_m(2 * M) == 0
    assert R.mod_m(2 ** 576 - 1) == 2 ** 240 - 2            # 2^576 = m + 2^240 - 1
    assert R.mod_m(2 ** 576) == 2 ** 240 - 1
    assert R.mod_m((M - 1) ** 2) == 1                         # (-1)^2
    # 2^1152 = (2^240 - 1)^2 = 2^480 - 2^241 + 1 < m
    assert R.mod_m(2 ** 1152 - 1) == 2 ** 480 - 2 ** 241
    assert R.mod_m(2 ** 1152) == 2 ** 480 - 2 ** 241 + 1


def test_multiply9x9_limbs():
    """Sec. 2.1: 18 output limbs; each 64-bit column sums its pair products."""
    rng = random.Random(11)
    for _ in range(100):
        x, y = rng.randrange(2 ** 576), rng.randrange(2 ** 576)
        xs = [(x >> (64 * i)) & (2 ** 64 - 1) for i in range(9)]
        ys = [(y >> (64 * i)) & (2 ** 64 - 1) for i in range(9)]
        cols = [0] * 19
        for i in range(9):
            for j in range(9):
                cols[i + j] += xs[i] * ys[j]
        acc, carry = 0, 0
        for k in range(18):
            t = cols[k] + carry
            acc |= (t & (2 ** 64 - 1)) << (64 * k)
            carry = t >> 64
        assert carry == 0
        assert R.multiply9x9(x, y) == acc


# --- seeding and skipping -------------------------------------------------------------
def test_skip_equals_single_advances():
    for p in (24, 2048):
        s = R.Stream(p, seed=3)
        t = R.Stream(p, seed=3)
        A = R.luxury_multiplier(p)
        X = t.X
        for n in range(1, 40):
            X = R.advance(X, A)
            s2 = R.Stream(p, X=s.X)
            s2.skip(n)
            assert s2.X == X


def test_skip_composes():
    rng = random.Random(17)
    for _ in range(10):
        n1, n2 = rng.randrange(2 ** 128), rng.randrange(2 ** 128)
        a = R.Stream(2048, seed=5)
        b = R.Stream(2048, seed=5)
        a.skip(n1)
        a.skip(n2)
        b.skip(n1 + n2)
        assert a.X == b.X


def test_seed_spacing_is_2_96_advances():
    p = 2048
    s1 = R.Stream(p, seed=1)
    s2 = R.Stream(p, seed=2)
    s1.skip(2 ** 96)
    assert s1.X == s2.X
    # seed 1 from the state 1 by square-and-multiply written out by hand
    A = R.luxury_multiplier(p)
    y = A
    for _ in range(96):
        y = y * y % R.M
    assert R.seed_lcg(1, p) == y
    # seeds start at 1 (seed 0 would be the unmoved state 1) and fit 64 bits
    for bad in (0, -1, 2 ** 64):
        with pytest.raises(ValueError):
            R.seed_lcg(bad, p)


def test_skip_keeps_position_and_matches_recurrence_blocks():
    p = 223
    s = R.Stream(p, seed=9)
    s.draw_u24(5)
    w, c = s.words(), s.c
    s.skip(3)
    assert s.pos == 5
    for _ in range(3):
        w, c = S.block(w, c, p)
    assert s.words() == w and s.c == c


# --- draw rule ---------------------------------------------------------------------------
def _blocks_from_recurrence(w, c, p, n_blocks):
    out = [list(w)]
    for _ in range(n_blocks - 1):
        w, c = S.block(w, c, p)
        out.append(list(w))
    return out


@pytest.mark.parametrize("p", [24, 389, 2048])
def test_u24_draws_are_recurrence_blocks(p):
    s = R.Stream(p, seed=4)
    blocks = _blocks_from_recurrence(s.words(), s.c, p, 5)
    got = s.draw_u24(24 * 5)
    assert got == [x for b in blocks for x in b]


@pytest.mark.parametrize("p", [24, 2048])
def test_f64_draws_pair_words_low_first(p):
    s = R.Stream(p, seed=6)
    blocks = _blocks_from_recurrence(s.words(), s.c, p, 4)
    got = s.draw_f64(12 * 4)
    want = [(b[2 * k] + (b[2 * k + 1] << 24)) * 2.0 ** -48 for b in blocks for k in range(12)]
    assert got == want
    for v in got:
        assert 0.0 <= v < 1.0 and (v * 2 ** 48).is_integer()


def test_f64_discards_odd_leftover_word():
    s = R.Stream(24, seed=8)
    blocks = _blocks_from_recurrence(s.words(), s.c, 24, 2)
    assert s.draw_u24(23) == blocks[0][:23]     # one word left in block 0
    v = s.draw_bits48(1)[0]                       # needs two: comes from block 1
    assert v == blocks[1][0] + (blocks[1][1] << 24)
    assert s.pos == 2


def test_double_conversion_closed_forms():
    assert R.f64_from_bits48(0) == 0.0
    assert R.f64_from_bits48(1) == 2.0 ** -48
    assert R.f64_from_bits48(2 ** 47) == 0.5
    assert R.f64_from_bits48(2 ** 48 - 1) == 1.0 - 2.0 ** -48
    assert R.f64_bits(R.f64_from_bits48(2 ** 48 - 1)) == 0x3FEFFFFFFFFFFFE0  # mantissa 2^52 - 2^5
    assert R.f64_bits(0.5) == 0x3FE0000000000000


def test_sum_hist_brute_force():
    vals = [0, 1, 2 ** 40 - 1, 2 ** 40, 2 ** 48 - 1, 5 * 2 ** 40 + 7]
    s, h = R.sum_hist48(vals)
    assert s == sum(vals)
    assert h[0] == 3 and h[1] == 1 and h[255] == 1 and h[5] == 1 and sum(h) == 6


# --- the C oracle's draw rule against the Python one -----------------------------------
@pytest.mark.parametrize("kind", [S.KIND_U24, S.KIND_F64, S.KIND_BITS48])
def test_c_draws_match_python(kind):
    p = 389
    streams = [R.Stream(p, seed=s) for s in range(1, 9)]
    for k, st in enumerate(streams):     # assorted start positions
        st.draw_u24(k * 3)
    words = np.array([st.words() for st in streams], dtype=np.uint32)
    carry = np.array([st.c for st in streams], dtype=np.uint32)
    pos = np.array([st.pos for st in streams], dtype=np.int32)
    n = 61
    got = S.draw_many(words, carry, pos, p, n, kind, threads=3)
    for k, st in enumerate(streams):
        if kind == S.KIND_U24:
            want = st.draw_u24(n)
        elif kind == S.KIND_F64:
            want = st.draw_f64(n)
        else:
            want = st.draw_bits48(n)
        assert list(got[k]) == want
        assert list(words[k]) == st.words() and carry[k] == st.c and pos[k] == st.pos


def test_c_sum_hist_matches_python():
    p = 2048
    streams = [R.Stream(p, seed=s) for s in range(1, 6)]
    words = np.array([st.words() for st in streams], dtype=np.uint32)
    carry = np.array([st.c for st in streams], dtype=np.uint32)
    pos = np.zeros(5, dtype=np.int32)
    sums, hist = S.sum_hist_many(words, carry, pos, p, 100, threads=2)
    all_vals = []
    for k, st in enumerate(streams):
        vals = st.draw_bits48(100)
        all_vals += vals
        assert int(sums[k]) == sum(vals)
    assert [int(h) for h in hist] == R.sum_hist48(all_vals)[1]


# --- golden regression vectors ------------------------------------------------------------
def test_golden_seed_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "seed_vectors.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p, s, kind, k, v = line.split()
            rows.append((int(p), int(s), kind, int(k), int(v, 16)))
    cache = {}
    for p, s, kind, k, v in rows:
        key = (p, s, kind)
        if key not in cache:
            st = R.Stream(p, seed=s)
            cache[key] = st.draw_u24(30) if kind == "u24" else [R.f64_bits(x) for x in st.draw_f64(15)]
        assert cache[key][k] == v, (p, s, kind, k)


# --- single-precision draws and skipping by values -------------------------------------
def test_f32_draws_are_the_u24_words_scaled():
    s = R.Stream(389, seed=12)
    t = R.Stream(389, seed=12)
    f = s.draw_f32_bits(100)
    u = t.draw_u24(100)
    import struct
    for fb, w in zip(f, u):
        x = struct.unpack("<f", struct.pack("<I", fb))[0]
        assert x * 2 ** 24 == w and 0.0 <= x < 1.0
    assert R.f32_bits_from24(0) == 0
    assert R.f32_bits_from24(1) == 0x33800000            # 2^-24
    assert R.f32_bits_from24(2 ** 23) == 0x3F000000      # 0.5
    assert R.f32_bits_from24(2 ** 24 - 1) == 0x3F7FFFFF  # 1 - 2^-24


def test_c_f32_draws_match_python():
    streams = [R.Stream(24, seed=s) for s in range(1, 5)]
    words = np.array([st.words() for st in streams], dtype=np.uint32)
    carry = np.array([st.c for st in streams], dtype=np.uint32)
    pos = np.zeros(4, dtype=np.int32)
    got = S.draw_many(words, carry, pos, 24, 50, S.KIND_F32, threads=2)
    for k, st in enumerate(streams):
        assert list(got[k].view(np.uint32)) == st.draw_f32_bits(50)


@pytest.mark.parametrize("need", [1, 2])
def test_skip_values_equals_drawing(need):
    rng = random.Random(31 + need)
    for _ in range(40):
        s = R.Stream(223, seed=rng.randrange(1, 100))
        t = R.Stream(223, X=s.X)
        s.draw_u24(rng.randrange(0, 30))
        t.pos = s.pos
        t.D, t.c = s.D, s.c
        n = rng.randrange(0, 200)
        (s.draw_bits48 if need == 2 else s.draw_u24)(n)
        t.skip_values(n, need)
        assert (t.D, t.c, t.pos) == (s.D, s.c, s.pos)


# --- Gaussian values (Box-Muller on pairs of doubles) ---------------------------------
def test_box_muller_closed_forms():
    import math
    assert R.box_muller(0.0, 0.3) == (0.0, 0.0)                      # u1 = 1: r = 0
    for k in (1, 2, 10, 48):
        d_a = 1.0 - 2.0 ** -k                                         # u1 = 2^-k exactly
        r = math.sqrt(2 * k * math.log(2.0))
        assert R.box_muller(d_a, 0.0) == pytest.approx((r, 0.0), rel=1e-15, abs=0)
        z = R.box_muller(d_a, 0.25)                                   # a quarter turn
        assert z[0] == 0.0 and z[1] == pytest.approx(r, rel=1e-15)
        z = R.box_muller(d_a, 0.5)
        assert z[0] == pytest.approx(-r, rel=1e-15) and z[1] == 0.0
        z = R.box_muller(d_a, 0.125)                                  # an eighth turn
        assert z[0] == pytest.approx(r / math.sqrt(2), rel=1e-15) and z[1] == pytest.approx(z[0], rel=1e-15)
    # the exact quarter-turn reduction against the plain formula
    rng = random.Random(31)
    for _ in range(10000):
        d = rng.randrange(2 ** 48) / 2 ** 48
        c, s = R.cos_sin_2pi(d)
        assert abs(c - math.cos(2 * math.pi * d)) < 2e-15 and abs(s - math.sin(2 * math.pi * d)) < 2e-15


def test_box_muller_invariants_and_vector_form():
    import math
    rng = random.Random(32)
    da = np.array([rng.randrange(2 ** 48) / 2 ** 48 for _ in range(5000)] + [0.0, 1 - 2 ** -48])
    db = np.array([rng.randrange(2 ** 48) / 2 ** 48 for _ in range(5002)])
    z0v, z1v = R.box_muller_many(da, db)
    for a, b, v0, v1 in zip(da, db, z0v, z1v):
        z0, z1 = R.box_muller(a, b)
        rr = -2.0 * math.log(1.0 - a)
        assert z0 * z0 + z1 * z1 == pytest.approx(rr, rel=1e-13, abs=1e-300)   # radius
        if rr > 1e-20:                                                          # angle
            ang = math.atan2(z1, z0) % (2 * math.pi)
            assert min(abs(ang - 2 * math.pi * b), 2 * math.pi - abs(ang - 2 * math.pi * b)) < 1e-12
        r = math.sqrt(rr)
        assert abs(v0 - z0) <= 2 ** -50 * (r + 1) and abs(v1 - z1) <= 2 ** -50 * (r + 1)


def test_exponential_closed_forms_and_distribution():
    import math
    assert R.exponential(0.0) == 0.0 and math.copysign(1, R.exponential(0.0)) == 1
    for k in (1, 2, 10, 24, 48):
        # 1 - d = 2^-k exactly, so x = k ln 2
        assert R.exponential(1.0 - 2.0 ** -k) == pytest.approx(k * math.log(2.0), rel=1e-15)
    assert R.exponential(0.5) == pytest.approx(math.log(2.0), rel=1e-15)
    # small d: -ln(1 - d) = d + d^2 / 2 + ..., and the distribution function at x gives d back
    for d in (2.0 ** -48, 2.0 ** -30, 3 * 2.0 ** -40):
        assert R.exponential(d) == pytest.approx(d + d * d / 2, rel=1e-15)
    rng = random.Random(33)
    for _ in range(2000):
        d = rng.randrange(2 ** 48) / 2 ** 48
        assert -math.expm1(-R.exponential(d)) == pytest.approx(d, rel=1e-14, abs=2 ** -52)
    st, ref = R.Stream(2048, seed=23), R.Stream(2048, seed=23)
    x = st.draw_exp(5)
    assert x == [R.exponential(d) for d in ref.draw_f64(5)] and st.state() == ref.state()
    # moments (mean 1, variance 1) and the Kolmogorov-Smirnov distance to 1 - e^-x
    n = 100000
    x = np.array(R.Stream(389, seed=24).draw_exp(n))
    assert x.min() >= 0
    assert abs(x.mean() - 1) < 5 / math.sqrt(n)
    assert abs(x.var() - 1) < 5 * math.sqrt(8 / n)        # the fourth central moment is 9
    xs = np.sort(x)
    cdf = -np.expm1(-xs)
    ks = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n)                        # 1 % critical value


def test_normal_draws_consume_pairs_and_look_gaussian():
    import math
    st, ref = R.Stream(2048, seed=21), R.Stream(2048, seed=21)
    z = st.draw_normal(7)                                 # odd: 8 doubles taken, 7 values
    d = ref.draw_f64(8)
    assert z == [v for k in range(0, 8, 2) for v in R.box_muller(d[k], d[k + 1])][:7]
    assert st.state() == ref.state()
    # moments and the Kolmogorov-Smirnov distance to the normal distribution
    n = 100000
    s = R.Stream(389, seed=22)
    x = np.array(s.draw_normal(n))
    assert abs(x.mean()) < 5 / math.sqrt(n)
    assert abs(x.var() - 1) < 5 * math.sqrt(2 / n)
    xs = np.sort(x)
    cdf = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in xs]))
    ks = max(np.max(np.arange(1, n + 1) / n - cdf), np.max(cdf - np.arange(n) / n))
    assert ks < 1.63 / math.sqrt(n)                        # 1 % critical value


# --- raw LCG doubles (comparison mode) ----------------------------------------------------
@pytest.mark.parametrize("p", [24, 389, 2048])
def test_raw52_draws_are_the_bits_of_the_recurrence_states(p):
    """The raw values of each refill reassemble the low 572 bits of the LCG state that the
    recurrence reaches after p more steps (X = D - floor(D / 2^336) + c of its window),
    low bits first, 11 per refill; the stream ends at the last refill's block, read
    position 24; and the values are below 2^52."""
    s = R.Stream(p, seed=9, pos=5)
    w, c = s.words(), s.c
    got = s.draw_raw52(11 * 3 + 4)      # four refills, the last one partly used
    assert len(got) == 37 and all(0 <= v < 2 ** 52 for v in got)
    for r in range(4):
        w, c = S.block(w, c, p)         # the recurrence's next block (p steps)
        X = R.pack_words(w) - (R.pack_words(w) >> 336) + c
        vals = got[11 * r: 11 * r + 11]
        assert sum(v << (52 * k) for k, v in enumerate(vals)) == X % 2 ** (52 * len(vals))
    assert s.words() == w and s.c == c and s.pos == 24
    # no values: no refill, nothing moves
    t = R.Stream(p, seed=9, pos=5)
    assert t.draw_raw52(0) == [] and t.pos == 5 and t.words() == R.Stream(p, seed=9).words()


def test_raw52_double_conversion_closed_forms():
    assert R.f64_from_bits52(0) == 0.0
    assert R.f64_from_bits52(1) == 2.0 ** -52
    assert R.f64_from_bits52(2 ** 51) == 0.5
    assert R.f64_from_bits52(2 ** 52 - 1) == 1.0 - 2.0 ** -52
