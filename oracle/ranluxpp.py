"""Big-integer oracle for RANLUX++ (Hahnfeld & Moneta, "A Portable Implementation of
RANLUX++", arXiv 2106.02504).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  The CUDA library never calls it,
and it shares no code, table or constant generator with the CUDA library.

Everything here is the plain definition, written with Python integers:

* the RANLUX subtract-with-borrow recurrence (base b = 2^24, lags r = 24, s = 10, with
  a borrow bit), which the paper builds on (Sec. 1, Sec. 2);
* its LCG form with modulus m = b^r - b^s + 1 = 2^576 - 2^240 + 1 (Sec. 2.2) and
  multiplier a = b^-1 mod m, raised to the luxury power p (Sec. 1: the generator is an
  LCG with a very large multiplier);
* the product of two 576-bit numbers (Sec. 2.1) as Python ``*`` and the reduction
  modulo m (Sec. 2.2) as Python ``%``: the remainder in [0, m) the paper's ``mod_m`` is
  required to return;
* the conversion from the LCG state back to 24 RANLUX numbers and the carry (Sec. 2.3):
  the digits of X/m in base 2^24, i.e. D = floor(2^576 X / m), with the carry fixed by
  the inverse map X = D - floor(D / 2^336) + c;
* 48-bit doubles in [0, 1) (Sec. 2.3), 24-bit integers (Sec. 2.4, ``IntRndm``) and
  24-bit single-precision floats w 2^-24 (RANLUX's own output format);
* seeding and skipping by exponentiation (Sec. 2.4) as Python ``pow``.

Readings where the paper is silent:

* seed s gives the LCG state a_p^(2^96 s) (the state 1 skipped by 2^96 s luxury
  advances; Sec. 2.5 mentions skipping 2^96 seed states), converted to RANLUX numbers
  with read position 0 and no extra advance;
* one draw position counts 24-bit words 0..24; a u24 draw takes the next word, a double
  takes the next two words w_k + 2^24 w_{k+1} (k = pos) and needs both in the current
  block, otherwise the generator advances first (a lone leftover word is discarded);
* skip(n) applies n luxury advances (A^n) to the LCG state and keeps the read position;
* seeds are 1 .. 2^64 - 1;
* Gaussian values come from consecutive pairs of the stream's doubles by the
  Box-Muller transform (Box and Muller, Ann. Math. Statist. 29, 1958), u1 = 1 - d_a so
  that ln u1 is finite; n values take 2 ceil(n / 2) doubles;
* raw LCG doubles (for comparison only) take 11 x 52 bits of each new LCG state, low
  bits first (Stream.draw_raw52).

Parity pins for every function are in ``tests/test_oracle_pins.py`` (SWB brute force,
closed forms, invariants and edge cases).
"""
from __future__ import annotations

import math
import struct

# --- Sec. 2.2: the modulus --------------------------------------------------------
BASE_BITS = 24
BASE = 1 << BASE_BITS          # b
LAG_R = 24                     # r
LAG_S = 10                     # s
M = BASE ** LAG_R - BASE ** LAG_S + 1   # m = b^r - b^s + 1 = 2^576 - 2^240 + 1
STATE_BITS = BASE_BITS * LAG_R  # 576
WORDS = LAG_R                   # 24 RANLUX numbers per block
MASK24 = BASE - 1
MASK48 = (1 << 48) - 1
SEED_SHIFT = 96                 # seed s = 2^96 s luxury advances from the state 1
RAW_BITS = 52                   # raw LCG doubles: 52 bits of the state each
RAW_PER_REFILL = STATE_BITS // RAW_BITS   # 11 per refill
MASK52 = (1 << RAW_BITS) - 1


# --- Sec. 1 / Sec. 2: the subtract-with-borrow recurrence -------------------------
def swb_step(window, carry):
    """One RANLUX step.  ``window`` lists the 24 live numbers, oldest first.

    x_n = x_{n-s} - x_{n-r} - c_{n-1} (mod b), and the new borrow c_n is 1 exactly when
    that difference was negative.  Returns the new window and borrow.
    """
    diff = window[LAG_R - LAG_S] - window[0] - carry
    new_carry = 1 if diff < 0 else 0
    return window[1:] + [diff % BASE], new_carry


def swb_steps(window, carry, n):
    """n recurrence steps (luxury p means p steps per delivered block of 24)."""
    for _ in range(n):
        window, carry = swb_step(window, carry)
    return window, carry


# --- Sec. 1: the equivalent LCG -----------------------------------------------------
def one_step_multiplier():
    """a = b^-1 mod m: one recurrence step multiplies the LCG state by a."""
    return pow(BASE, -1, M)


def luxury_multiplier(p):
    """A = a^p mod m: one LCG advance at luxury level p (p recurrence steps)."""
    return pow(one_step_multiplier(), p, M)


def multiply9x9(x, y):
    """Sec. 2.1: the full 1152-bit product of two 576-bit numbers."""
    return x * y


def mod_m(v):
    """Sec. 2.2: the remainder of v modulo m, always in [0, m)."""
    return v % M


def advance(X, A):
    """One LCG step X <- A X mod m (Sec. 2, Sec. 2.1-2.2)."""
    return mod_m(multiply9x9(A, X))


# --- Sec. 2.3: conversion between the LCG state and RANLUX numbers -----------------
def pack_words(words):
    """D = sum_i w_i 2^(24 i), w_0 the oldest number."""
    return sum(w << (BASE_BITS * i) for i, w in enumerate(words))


def unpack_words(D):
    return [(D >> (BASE_BITS * i)) & MASK24 for i in range(WORDS)]


def to_ranlux(X):
    """LCG state X in [0, m) -> (D, c): D = floor(2^576 X / m), the base-2^24 digits of
    X/m, and the borrow c that makes to_lcg(D, c) == X."""
    D = (X << STATE_BITS) // M
    c = X - D + (D >> (BASE_BITS * (LAG_R - LAG_S)))
    return D, c


def to_lcg(D, c):
    """(D, c) -> X = D - floor(D / 2^336) + c, 336 = 24 (r - s) bits."""
    return D - (D >> (BASE_BITS * (LAG_R - LAG_S))) + c


# --- Sec. 2.3: output formats -------------------------------------------------------
def f64_from_bits48(v):
    """48 random bits -> a double in [0, 1): v * 2^-48, exact for v < 2^53."""
    return float(v) * 2.0 ** -48



def cos_sin_2pi(d):
    """(cos 2 pi d, sin 2 pi d) for a double d in [0, 1): 4d is exact, so it splits
    exactly into q quarter turns (q = round(4d)) and a rest f in [-1/2, 1/2]; the angle
    (pi / 2) f is at most pi / 4, where math.cos and math.sin are accurate to about an
    ulp, and the quarter turns are exact sign and order changes."""
    t = 4.0 * d
    q = int(round(t))
    f = t - q
    th = (math.pi / 2.0) * f
    c, s = math.cos(th), math.sin(th)
    return [(c, s), (-s, c), (-c, -s), (s, -c)][q % 4]


def box_muller(d_a, d_b):
    """Box and Muller (1958): two standard Gaussian values from two doubles in [0, 1):
    u1 = 1 - d_a in (0, 1] (exact for 48-bit doubles), r = sqrt(-2 ln u1), then
    (r cos 2 pi d_b, r sin 2 pi d_b)."""
    u1 = 1.0 - d_a
    r = math.sqrt(-2.0 * math.log(u1))
    c, s = cos_sin_2pi(d_b)
    return r * c, r * s


def box_muller_many(d_a, d_b):
    """box_muller over numpy arrays of pairs (the same steps with numpy's log, sqrt, cos
    and sin); returns the two arrays of values."""
    import numpy as np
    d_a = np.asarray(d_a, dtype=np.float64)
    d_b = np.asarray(d_b, dtype=np.float64)
    r = np.sqrt(-2.0 * np.log(1.0 - d_a))
    t = 4.0 * d_b
    q = np.rint(t)
    th = (math.pi / 2.0) * (t - q)
    c, s = np.cos(th), np.sin(th)
    qi = q.astype(np.int64) % 4
    return r * np.choose(qi, [c, -s, -c, s]), r * np.choose(qi, [s, c, -s, -c])


def exponential(d):
    """Exponential value with rate 1 by inversion of its distribution function
    F(x) = 1 - e^-x: x = -ln(1 - d) for a double d in [0, 1) (1 - d is exact for 48-bit
    doubles; d = 0 gives 0)."""
    return 0.0 - math.log(1.0 - d)


def f64_from_bits52(v):
    """52 raw LCG bits -> v 2^-52 in [0, 1), exact."""
    return float(v) * 2.0 ** -52


def f64_bits(x):
    """IEEE-754 binary64 bit pattern of a Python float."""
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def f32_bits_from24(w):
    """One 24-bit number -> the binary32 bit pattern of w 2^-24 in [0, 1) (exact: w has
    at most 24 significant bits)."""
    return struct.unpack("<I", struct.pack("<f", float(w) * 2.0 ** -24))[0]


# --- Sec. 2.4: seeding and skipping -------------------------------------------------
def seed_lcg(seed, p):
    """LCG state of seed s: the state 1 skipped by 2^96 s luxury advances.  Seeds are
    1 .. 2^64 - 1; seed 0 would leave the state 1 itself and is rejected."""
    if not 1 <= seed < 1 << 64:
        raise ValueError("seed must be in [1, 2^64)")
    return pow(luxury_multiplier(p), seed << SEED_SHIFT, M)


class Stream:
    """One generator: RANLUX numbers D, borrow c, read position (in 24-bit words) and
    the luxury level p.  Mirrors the paper's final design (Sec. 2): the packed RANLUX
    numbers and the carry are the state, the LCG form is rebuilt to advance."""

    def __init__(self, p, seed=None, X=None, pos=0, A=None):
        self.p = p
        self.A = luxury_multiplier(p) if A is None else A
        if X is None:
            X = seed_lcg(seed, p) if seed is not None else 1
        self.D, self.c = to_ranlux(X)
        self.pos = pos

    # state as the LCG number
    @property
    def X(self):
        return to_lcg(self.D, self.c)

    def words(self):
        return unpack_words(self.D)

    def _refill(self):
        self.D, self.c = to_ranlux(advance(self.X, self.A))
        self.pos = 0

    def draw_u24(self, n):
        out = []
        for _ in range(n):
            if self.pos + 1 > WORDS:
                self._refill()
            out.append((self.D >> (BASE_BITS * self.pos)) & MASK24)
            self.pos += 1
        return out

    def draw_bits48(self, n):
        out = []
        for _ in range(n):
            if self.pos + 2 > WORDS:
                self._refill()
            out.append((self.D >> (BASE_BITS * self.pos)) & MASK48)
            self.pos += 2
        return out

    def draw_f64(self, n):
        return [f64_from_bits48(v) for v in self.draw_bits48(n)]

    def draw_normal(self, n):
        """n Gaussian values: Box-Muller on consecutive pairs of 2 ceil(n / 2) doubles."""
        d = self.draw_f64(n + (n & 1))
        out = []
        for k in range(0, len(d), 2):
            out.extend(box_muller(d[k], d[k + 1]))
        return out[:n]

    def draw_exp(self, n):
        """n exponential values, one double each."""
        return [exponential(d) for d in self.draw_f64(n)]

    def draw_f32_bits(self, n):
        """Single-precision draws: one number each, w 2^-24 (the 24-bit RANLUX output)."""
        return [f32_bits_from24(w) for w in self.draw_u24(n)]

    def draw_raw52(self, n):
        """Raw LCG doubles (Sec. 2.3 names this form, Sibidanov's, only to replace it by
        the RANLUX numbers: its top bits are biased towards 0 because X < m; for
        comparison only), as 52-bit integers v (the double is v 2^-52).  Each refill of
        the LCG state gives 11 values, v_k = (X >> 52 k) mod 2^52 for k = 0 .. 10 of the
        new state X, low bits first; the top 4 bits of X are not used.  A draw of n
        values starts with a refill, takes ceil(n / 11) of them, discards the values of
        the last one past n, and leaves the stream at the end of that block (read
        position 24); n = 0 changes nothing."""
        out = []
        X = self.X
        while len(out) < n:
            X = advance(X, self.A)
            out.extend((X >> (RAW_BITS * k)) & MASK52 for k in range(RAW_PER_REFILL))
        if n:
            self.D, self.c = to_ranlux(X)
            self.pos = WORDS
        return out[:n]

    def skip_values(self, n, per_value_words):
        """Move as if n values taking per_value_words numbers each had been drawn."""
        pos, need = self.pos, per_value_words
        room = (WORDS - pos) // need if pos + need <= WORDS else 0
        if n <= room:
            self.pos = pos + n * need
            return
        rest = n - room
        per = WORDS // need
        blocks = -(-rest // per)
        X = pow(self.A, blocks, M) * self.X % M
        self.D, self.c = to_ranlux(X)
        self.pos = (rest - (blocks - 1) * per) * need

    def skip(self, n):
        """Apply n luxury advances without producing output; the position is kept."""
        X = pow(self.A, n, M) * self.X % M
        self.D, self.c = to_ranlux(X)

    def state(self):
        """(D as nine little-endian 64-bit limbs, c, pos, p)."""
        return ([(self.D >> (64 * i)) & ((1 << 64) - 1) for i in range(9)],
                self.c, self.pos, self.p)


def sum_hist48(values48):
    """Exact integer sum of 48-bit values and the 256-bin histogram of their top 8 bits
    (the fused consumer of the GPU throughput benchmark, Sec. 4.2, with an exact sum)."""
    hist = [0] * 256
    for v in values48:
        hist[v >> 40] += 1
    return sum(values48), hist
