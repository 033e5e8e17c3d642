"""The crafted inputs of tests/rare_paths.py reach the rare carry branches they are
built for (checked on the CPU against the plain models of each step's intermediate
value), so that the GPU parity tests that use them cover those branches."""
import random

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
