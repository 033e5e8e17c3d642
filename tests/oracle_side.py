"""Oracle-side helpers for the parity tests: expected states and outputs computed only
with ``oracle/`` (Python big integers for the LCG form, the C recurrence for volume)."""
from __future__ import annotations

import numpy as np

from oracle import ranluxpp as R
from oracle import swb_lib as S

MASK64 = (1 << 64) - 1


def limbs64(v, n):
    return [(v >> (64 * k)) & MASK64 for k in range(n)]


def from_limbs64(arr):
    return sum(int(x) << (64 * k) for k, x in enumerate(arr))


def seeded_X(seeds, p):
    """LCG states of the given seeds (dict seed -> X); consecutive runs share work."""
    A = R.luxury_multiplier(p)
    B = pow(A, 1 << R.SEED_SHIFT, R.M)
    out = {}
    prev_seed, prev_X = None, None
    for s in sorted(set(int(x) for x in seeds)):
        if prev_seed is not None and s == prev_seed + 1:
            X = prev_X * B % R.M
        else:
            X = pow(B, s, R.M)
        out[s] = X
        prev_seed, prev_X = s, X
    return out


class StreamSet:
    """Oracle copies of many streams as recurrence windows (for the C oracle)."""

    def __init__(self, Xs, p, pos=None):
        n = len(Xs)
        self.p = p
        self.words = np.zeros((n, 24), dtype=np.uint32)
        self.carry = np.zeros(n, dtype=np.uint32)
        self.pos = np.zeros(n, dtype=np.int32) if pos is None else np.array(pos, dtype=np.int32)
        for i, X in enumerate(Xs):
            D, c = R.to_ranlux(X)
            self.words[i] = R.unpack_words(D)
            self.carry[i] = c

    @classmethod
    def from_seeds(cls, seeds, p):
        xs = seeded_X(seeds, p)
        return cls([xs[int(s)] for s in seeds], p)

    def draw(self, count, kind):
        return S.draw_many(self.words, self.carry, self.pos, self.p, count, kind)

    def draw_ragged(self, counts, kind):
        """counts[i] values from stream i (in place, one stream at a time); a list of arrays."""
        out = []
        for i in range(self.words.shape[0]):
            one = StreamSet.__new__(StreamSet)
            one.p = self.p
            one.words, one.carry, one.pos = self.words[i:i + 1], self.carry[i:i + 1], self.pos[i:i + 1]
            out.append(one.draw(int(counts[i]), kind)[0])
        return out

    def sum_hist(self, count):
        return S.sum_hist_many(self.words, self.carry, self.pos, self.p, count)

    def D(self, i):
        return R.pack_words(int(w) for w in self.words[i])

    def state_records(self):
        """(n, 11) uint64 rows laid out like struct rlxpp_state."""
        n = self.words.shape[0]
        rec = np.zeros((n, 11), dtype=np.uint64)
        for i in range(n):
            rec[i, :9] = limbs64(self.D(i), 9)
            rec[i, 9] = int(self.carry[i]) | (int(self.pos[i]) << 32)
            rec[i, 10] = self.p
        return rec


def conversion_edge_states(rng, k=40):
    """LCG states at the corners of the conversion D = floor(2^576 X / m) (Sec. 2.3):
    X = ceil(q m / (2^240 - 1)) puts X (2^240 - 1) in [q m, q 2^576), where the quotient
    by m exceeds the quotient by 2^576 by one; and states whose shifted copy
    (X << 240) mod 2^576 agrees with X in bits 480..575, where comparing the top limbs
    alone cannot decide the borrow."""
    M = R.M
    out = []
    qs = [1, 2, 3, 2 ** 32, 2 ** 100 + 7, 2 ** 239, 2 ** 240 - 2] + [rng.randrange(1, 2 ** 240 - 1) for _ in range(k)]
    for q in qs:
        out.append(-(-q * M // (2 ** 240 - 1)))
    top = ((1 << 96) - 1) << 480
    for _ in range(k):
        X = rng.randrange(1, M)
        S = (X << 240) % 2 ** 576
        X2 = (X & ~top) | (S & top)
        if 0 < X2 < M:
            out.append(X2)
        X3 = (X2 - (1 << 480)) % M   # one below in limb 15: the top limbs of S - X all ones
        if X3:
            out.append(X3)
    return [x for x in out if 0 < x < M]


def normals_expected(doubles, n):
    """Gaussian values the draw rule gives from each row's doubles (2 ceil(n / 2) of
    them), with a per-value tolerance: (want, tol), both (rows, n) float64.  The device
    computes ln, sqrt, cos and sin with its own fixed-point integer routines and rounds
    each Gaussian value once: it lies within half an ulp plus 2^-56 r of the exact value
    (ln to a relative 2^-61, the square root to a relative 2^-59, cos and sin to an
    absolute 2^-59, all before the final rounding).  The oracle uses Python's double
    log, sqrt, cos and sin after an exact quarter-turn reduction, so it is within a few
    ulp of r.  With r <= sqrt(96 ln 2) < 8.2, an ulp of a value is at most 2^-52 r, so
    the two sides differ by well under 2^-49 (r + 1), the tolerance used here."""
    d = np.asarray(doubles, dtype=np.float64)
    da, db = d[:, 0::2], d[:, 1::2]
    z0, z1 = R.box_muller_many(da, db)
    want = np.empty_like(d)
    want[:, 0::2], want[:, 1::2] = z0, z1
    r = np.sqrt(-2.0 * np.log(1.0 - da))
    tol = np.repeat(2.0 ** -49 * (r + 1.0), 2, axis=1)
    return want[:, :n], tol[:, :n]


def exponentials_expected(doubles):
    """Exponential values x = -ln(1 - d) from each double, with a per-value tolerance:
    (want, tol).  The device computes -ln with its own fixed-point integer routine
    (relative error below 2^-61 before its one final rounding), so its value lies within
    half an ulp plus 2^-60 x of the exact one; numpy's log is within about an ulp.  An ulp
    of x is at most 2^-52 x, so the two differ by well under 2^-51 x; the tolerance
    2^-50 (x + 1) leaves a factor of two and an absolute floor for x near 0."""
    d = np.asarray(doubles, dtype=np.float64)
    want = 0.0 - np.log(1.0 - d)
    return want, 2.0 ** -50 * (want + 1.0)


def records_from_windows(words, carry, pos, p):
    """(n, 11) uint64 state records (struct rlxpp_state: the 24 numbers packed as 9
    little-endian 64-bit limbs, carry | pos << 32, p) from oracle windows, vectorised:
    every 8 numbers (192 bits) fill 3 limbs."""
    w = np.asarray(words, dtype=np.uint64)
    n = w.shape[0]
    rec = np.zeros((n, 11), dtype=np.uint64)
    for g in range(3):
        x = [w[:, 8 * g + k] for k in range(8)]
        rec[:, 3 * g] = x[0] | (x[1] << np.uint64(24)) | ((x[2] & np.uint64(0xFFFF)) << np.uint64(48))
        rec[:, 3 * g + 1] = ((x[2] >> np.uint64(16)) | (x[3] << np.uint64(8)) | (x[4] << np.uint64(32))
                             | ((x[5] & np.uint64(0xFF)) << np.uint64(56)))
        rec[:, 3 * g + 2] = (x[5] >> np.uint64(8)) | (x[6] << np.uint64(16)) | (x[7] << np.uint64(40))
    rec[:, 9] = np.asarray(carry, dtype=np.uint64) | (np.asarray(pos, dtype=np.uint64) << np.uint64(32))
    rec[:, 10] = p
    return rec


def weighted_checksum(values):
    """sum_j v_j (2 j + 1) mod 2^64 along the last axis (v as unsigned 64-bit bit
    patterns).  The weights are odd, hence invertible mod 2^64, so any single changed
    value changes the sum, and values out of order change it unless their differences
    cancel by chance."""
    v = np.asarray(values)
    v = v.view(np.uint64) if v.dtype.itemsize == 8 else v.astype(np.uint64)
    w = np.arange(1, 2 * v.shape[-1], 2, dtype=np.uint64)
    return (v * w).sum(axis=-1, dtype=np.uint64)


def skipped_states(job):
    """For a process pool: X_i A^d_i mod m for (X_i, d_i) pairs at luxury p, by pow."""
    p, pairs = job
    A = R.luxury_multiplier(p)
    return [pow(A, d, R.M) * X % R.M for X, d in pairs]
