"""Host logic of the serving loop without a GPU: the stream-cursor arithmetic against the
oracle's draw rule, and the first-fit arena (alignment, coalescing, exhaustion) against a
brute-force model of the free bytes."""
import random

import numpy as np

from oracle import ranluxpp as R
from paper_2106_02504_gb300.serve import Arena, advance_cursor


def test_cursor_arithmetic_matches_oracle_rule():
    st = R.Stream(24, seed=3)
    block, pos = 0, 0
    rng = np.random.Generator(np.random.PCG64(9))
    for _ in range(300):
        kind, count = int(rng.integers(0, 2)), int(rng.integers(0, 60))
        (st.draw_f64 if kind == 1 else st.draw_u24)(count)
        block, pos = advance_cursor(block, pos, kind, count)
        assert pos == st.pos
        # the stream's LCG state sits `block` advances after the seeded state
        assert pow(R.luxury_multiplier(24), block, R.M) * R.seed_lcg(3, 24) % R.M == st.X


def test_arena_first_fit_and_coalescing():
    size = 1 << 16
    a = Arena(size)
    rng = random.Random(5)
    live = {}                       # offset -> length
    free = np.ones(size, dtype=bool)
    for step in range(3000):
        if live and (rng.random() < 0.45 or a.used > size * 0.9):
            off = rng.choice(list(live))
            n = live.pop(off)
            a.release(off, n)
            free[off:off + n] = True
        else:
            want = rng.randrange(1, 5000)
            got = a.alloc(want)
            need = -(-want // 256) * 256
            # first fit: the lowest 256-aligned run of `need` free bytes, if any
            first = None
            for off in range(0, size - need + 1, 256):
                if free[off:off + need].all():
                    first = off
                    break
            if got is None:
                assert first is None, step
                continue
            off, n = got
            assert n == need and off == first and off % 256 == 0, step
            free[off:off + n] = False
            live[off] = n
        assert a.used == size - int(free.sum())
        # the free list is sorted, coalesced and covers exactly the free bytes
        prev_end = -1
        for off, ln in a.free:
            assert off > prev_end and ln > 0
            prev_end = off + ln
            assert free[off:off + ln].all()
        assert sum(ln for _, ln in a.free) == int(free.sum())
    for off, n in list(live.items()):
        a.release(off, n)
    assert a.free == [(0, size)] and a.used == 0


def test_arena_rounds_pool_and_requests_to_granules():
    """A pool that is not a whole number of 256-byte granules is used down to the last
    whole one, so a request that fits the pool only before rounding is refused instead
    of waiting forever."""
    a = Arena(1000 // 256 * 256)
    assert a.alloc(768) == (0, 768) and a.alloc(1) is None
    a.release(0, 768)
    assert a.alloc(769) is None and a.free == [(0, 768)]
