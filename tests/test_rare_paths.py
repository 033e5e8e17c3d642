"""The crafted inputs of tests/rare_paths.py reach the rare carry branches they are
built for (checked on the CPU against the plain models of each step's intermediate
value), so that the GPU parity tests that use them cover those branches."""
import random

import pytest

from oracle import ranluxpp as R
from tests import rare_paths as RP


def test_mod_m_inputs_reach_every_carry():
    ps = RP.mod_m_carry_inputs(random.Random(26))
    assert all(0 <= p < 2 ** 1152 for p in ps)
    folds = [RP.mod_m_fold_carries(p) for p in ps]
    assert sum(f[0] for f in folds) >= 24      # past limb 7 in the first fold
    assert sum(f[1] for f in folds) >= 24      # past limb 8
    assert sum(f[2] for f in folds) >= 24      # out of limb 17: the second fold
    H = [p >> 576 for p in ps]
    assert sum((h % 2 ** 256) + (h >> 336) >= 2 ** 256 for h in H) >= 24   # H + H1 past limb 7
    assert sum((h % 2 ** 320) + (h >> 336) >= 2 ** 320 for h in H) >= 12   # ... and past limb 9


def test_conversion_states_carry():
    xs = RP.conversion_carry_states(random.Random(27))
    q = [x * (2 ** 240 - 1) // R.M for x in xs]
    assert all(0 < x < R.M for x in xs)
    assert sum((x % 2 ** 256) + qq >= 2 ** 256 for x, qq in zip(xs, q)) >= 72
    assert sum((x % 2 ** 288) + qq >= 2 ** 288 for x, qq in zip(xs, q)) >= 24
    assert sum(RP.conversion_borrow_runs(x) for x in xs) >= 24


def test_tc_model_and_crafted_operands():
    rng = random.Random(7)
    A = R.luxury_multiplier(2048)
    for _ in range(20):   # the model is congruent to the product and its top limb in range
        x = rng.randrange(2 ** 576)
        v = RP.tc_assembled(x, A)
        assert v % R.M == A * x % R.M and 16128 <= v >> 576 <= 34489
    hits = RP.tc_limb8_carry_inputs(A, random.Random(2148))
    assert hits and all(RP.tc_fold_carries(x, A)[0] for x in hits)
    assert all(RP.tc_fold_carries(x, A)[1] for x in RP.tc_above_m_inputs(A))


def _tc_epilogue_common_path(v):
    """The tensor draw kernels' epilogue on its common path, restated on Python integers
    limb by limb as the kernel computes it from the assembled value v: the fold with
    limbs 1..6 taken unchanged (right when limb 0 does not borrow) and its carry stopped
    at limb 8, and the conversion's quick quotient with its carry stopped at limb 7.
    Returns (X, D, rare), rare being the kernel's test for redoing both exactly."""
    T, Xa = v >> 576, v % RP.B576
    a = [(Xa >> (32 * k)) & 0xFFFFFFFF for k in range(18)]
    b0 = a[0] < T
    s78 = a[7] + (a[8] << 32) + (T << 16)
    c9 = s78 >> 64
    limbs = [(a[0] - T) % (1 << 32)] + a[1:7] + [s78 & 0xFFFFFFFF, (s78 >> 32) & 0xFFFFFFFF] + a[9:]
    X = sum(l << (32 * k) for k, l in enumerate(limbs))
    S = (X << 240) % RP.B576
    top = (S >> 480) - (X >> 480)              # limbs 15..17 of S - X, no borrow from below
    borrow = 1 if top < 0 else 0
    t = top % (1 << 96)
    q0 = (X >> 336) & 0xFFFFFFFF
    # q = (X >> 336) - borrow, the borrow taken from its lowest limb alone
    s8 = (X % RP.B256) + (q0 - borrow) % (1 << 32) + ((X >> 368) << 32)
    c8 = s8 >> 256
    D = (X >> 256 << 256) | (s8 % RP.B256)
    rare = (b0 or c9 or c8 or limbs[17] == 0xFFFFFFFF or t == (1 << 96) - 1 or t == 0 or q0 < borrow)
    return X, D, rare


def _assembled_x(x, A):
    return RP.tc_assembled(x, A)


def _assembled_d(x, A):
    D, c = R.to_ranlux(x)
    return RP.tc_assembled_d(D, c, A)


@pytest.mark.parametrize("form", ["x", "d"])
def test_tc_epilogue_common_path_is_exact(form):
    """Wherever the kernel's test lets the common path stand, its X and D equal A x mod m
    and floor(2^576 X / m), for operand rows holding X (the draw kernels with per-stream
    counts) and holding D and c (the fused, value and request kernels); the crafted
    operands all take the rare branch."""
    assembled = _assembled_x if form == "x" else _assembled_d
    rng = random.Random(8 if form == "x" else 9)
    for p in (24, 2048):
        A = R.luxury_multiplier(p)
        common = 0
        for _ in range(4000):
            x = rng.randrange(1, R.M)
            X, D, rare = _tc_epilogue_common_path(assembled(x, A))
            if not rare:
                common += 1
                assert X == A * x % R.M
                assert D == R.to_ranlux(X)[0]
        assert common >= 3990
    A = R.luxury_multiplier(2048)
    Ainv = pow(A, -1, R.M)
    if form == "x":
        crafted = RP.tc_limb8_carry_inputs(A, random.Random(2548)) + RP.tc_above_m_inputs(A)[1:]
    else:
        crafted = (RP.tc_d_borrow_states(A, random.Random(2748)) + RP.tc_d_limb8_carry_states(A, random.Random(2848))
                   + RP.tc_d_above_m_states(A))
    crafted += [Ainv * y % R.M for y in RP.conversion_carry_states(random.Random(2648), k=8)]
    assert all(_tc_epilogue_common_path(assembled(x, A))[2] for x in crafted)


def test_tc_d_crafted_states_reach_their_cases():
    """The crafted states for operand rows holding D and c reach the case each is built
    for: a borrow out of limb 0 of the fold, a carry out of limb 8, the final correction."""
    for p in (389, 2048):
        A = R.luxury_multiplier(p)
        for want, states in ((0, RP.tc_d_borrow_states(A, random.Random(p))),
                             (1, RP.tc_d_limb8_carry_states(A, random.Random(p + 1), want=2)),
                             (2, RP.tc_d_above_m_states(A))):
            assert states
            for X in states:
                assert 0 < X < R.M
                D, c = R.to_ranlux(X)
                assert R.to_lcg(D, c) == X
                assert RP.tc_fold_cases_d(D, c, A)[want]
