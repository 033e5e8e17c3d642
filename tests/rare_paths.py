"""Inputs that drive the device arithmetic into its rare carry branches.

The reduction mod m (Sec. 2.2), the conversion to RANLUX numbers (Sec. 2.3) and the fold
of the tensor-core column sums each propagate a carry past limb 7 or limb 8 only in a
branch that random inputs reach with probability 2^-13 to 2^-32.  These helpers build
inputs that reach those branches from a plain model of each step's intermediate value
(integers only, written from the step's definition).  They choose inputs; every expected
value still comes from the oracle."""
from __future__ import annotations

import bisect
import random

from oracle import ranluxpp as R

M = R.M
B256, B288, B576 = 1 << 256, 1 << 288, 1 << 576


# ---- reduction mod m: p = L + H 2^576 ----------------------------------------------
def _mod_m_offset(H):
    """K with R = L + K for the reduction's sum R = L + S 2^240 + (2m - V), where
    H1 = H >> 336, S = (H mod 2^336) + H1 and V = H + H1."""
    H1 = H >> 336
    S = (H & ((1 << 336) - 1)) + H1
    V = H + H1
    return (2 * M - V) + (S << 240)


def mod_m_carry_inputs(rng: random.Random, k: int = 24):
    """Products p < 2^1152 whose reduction carries out of limb 7 (and further) in each
    of its chains: H with limbs 0..7 (and 8, 9) all ones, so that H + H1 carries into
    limb 8 (and 10); and L chosen so that the sum R before the first fold has its low
    256, 288 or all 576 bits set, so that the fold carries past limb 7, past limb 8, or
    out of limb 17 (the second fold)."""
    out = []
    for _ in range(k):
        top = rng.randrange(1, 1 << 320)
        out.append(((top << 256) | (B256 - 1)) << 576 | rng.randrange(B576))
        top = rng.randrange(1, 1 << 256)
        out.append(((top << 320) | ((1 << 320) - 1)) << 576 | rng.randrange(B576))
    for _ in range(k):
        H = rng.randrange(B576)
        K = _mod_m_offset(H)
        for target in (rng.randrange(1 << 320) << 256 | (B256 - 1),
                       rng.randrange(1 << 288) << 288 | (B288 - 1),
                       B576 - 1,
                       B576 - 1 - rng.randrange(1 << 200)):
            L = (target - K) % B576
            out.append(H << 576 | L)
    return out


def mod_m_fold_carries(p):
    """(carry out of limb 7, carry out of limb 8, carry out of limb 17) of the first fold
    for the product p, from the model above."""
    L, H = p % B576, p >> 576
    Rv = L + _mod_m_offset(H)
    t, lo = Rv >> 576, Rv % B576
    add = t * ((1 << 240) - 1)
    return ((lo % B256) + add >= B256, (lo % B288) + add >= B288, lo + add >= B576)


# ---- conversion X -> D = X + q, q = floor(X (2^240 - 1) / m) -----------------------
def conversion_carry_states(rng: random.Random, k: int = 24):
    """States 0 < X < m whose limbs 0..7 (and 8, 9) are all ones, so that X + q carries
    out of limb 7 (and further) whenever q >= 1, and states whose q takes its borrow
    past its lowest limb."""
    out = []
    for _ in range(k):
        for low_bits in (256, 288, 320):
            top = rng.randrange(1, (M >> low_bits) - 1)
            X = (top << low_bits) | ((1 << low_bits) - 1)
            assert 0 < X < M
            out.append(X)
        # the lowest limb of X >> 336 zero while [(X << 240) mod 2^576 < X] = 1: the
        # borrow of q = (X >> 336) - [...] runs past that limb
        top = rng.randrange(1 << 180, M >> 368)
        out.append(top << 368 | rng.randrange(1 << 300))
    return out


def conversion_borrow_runs(X):
    """Whether q = (X >> 336) - [(X << 240) mod 2^576 < X] borrows past its lowest limb."""
    b = 1 if ((X << 240) % B576) < X else 0
    return ((X >> 336) & 0xFFFFFFFF) < b


# ---- the tensor-core product: column sums of the bytes of X against R_j ------------
C_BIAS = sum(0x3F003F000000 << (32 * t) for t in range(18))


def tc_assembled(x, A):
    """The value the tensor-core epilogue assembles from the 72 column sums before its
    fold: sum_j x_j R_j (x_j the bytes of x, R_j = A 2^(8j) mod m) plus the accumulator
    bias C and its cancelling constant E = -C mod m.  It is congruent to A x mod m."""
    E = (-C_BIAS) % M
    return C_BIAS + E + sum(((x >> (8 * j)) & 0xFF) * (A * pow(2, 8 * j, M) % M) for j in range(72))


def tc_fold_carries(x, A):
    """(carry out of limb 8, value >= m after the folds) for the tensor-core epilogue."""
    v = tc_assembled(x, A)
    T, lo = v >> 576, v % B576
    add = T * ((1 << 240) - 1)
    past8 = (lo % B288) + add >= B288
    f = lo + add
    if f >= B576:
        f = f - B576 + (1 << 240) - 1
    return past8, f >= M


def tc_limb8_carry_inputs(A, rng: random.Random, want: int = 4):
    """Operands x whose assembled value carries out of limb 8 in the fold, found by
    meeting in the middle over the low six bytes of x (2^18 choices on each side;
    about 2^-33 of the pairs qualify, so a handful are found)."""
    base = rng.randrange(B576) & ~((1 << 48) - 1)
    E = (-C_BIAS) % M
    Rj = [A * pow(2, 8 * j, M) % M for j in range(72)]
    v0 = C_BIAS + E + sum(((base >> (8 * j)) & 0xFF) * Rj[j] for j in range(72))
    width = 16128 << 240  # the fold adds at least this much (the top limb is >= 16128)

    def side(j0):
        vals = []
        for a in range(256):
            for b in range(256):
                for c in range(4):
                    vals.append(((a * Rj[j0] + b * Rj[j0 + 1] + c * Rj[j0 + 2]) % B288, (a, b, c)))
        return vals

    left = [((v0 + d) % B288, t) for d, t in side(0)]
    right = sorted(side(3))
    keys = [r[0] for r in right]
    found = []
    for a_val, ta in left:
        lo = (B288 - width - a_val) % B288
        hi = (B288 - a_val) % B288
        spans = [(lo, hi)] if lo < hi else [(lo, B288), (0, hi)]
        for s, e in spans:
            for idx in range(bisect.bisect_left(keys, s), bisect.bisect_left(keys, e)):
                tb = right[idx][1]
                x = base | ta[0] | ta[1] << 8 | ta[2] << 16 | tb[0] << 24 | tb[1] << 32 | tb[2] << 40
                if tc_fold_carries(x, A)[0]:
                    found.append(x)
        if len(found) >= want:
            break
    return found


def tc_above_m_inputs(A, rs=(0, 1, 2, 5, 1 << 100, (1 << 239) + 7, (1 << 240) - 3)):
    """Operands x = A^-1 r mod m whose product r is below 2^240 - 1, so that the folded
    value can be r + m, which needs the final correction."""
    Ainv = pow(A, -1, M)
    return [Ainv * r % M for r in rs]


# ---- the tensor-core product on operand rows that hold D and c ---------------------
# The fused, value and request kernels feed the product the RANLUX numbers D (72 bytes)
# and the borrow c of a state instead of X = D - floor(D / 2^336) + c.  Byte j of D
# stands for 2^(8j), less 2^(8(j - 42)) for j >= 42, so row j of their matrix holds
# R'_j = R_j - R_(j-42) mod m and a further row holds A against c.

def _rows_d(A):
    R = [A * pow(2, 8 * j, M) % M for j in range(72)]
    return [(R[j] - R[j - 42]) % M if j >= 42 else R[j] for j in range(72)]


def tc_assembled_d(D, c, A):
    """The value the epilogue assembles before its fold when the operand row holds D and
    c: sum_j d_j R'_j + c A plus the bias C and E = -C mod m.  Congruent to A X mod m."""
    E = (-C_BIAS) % M
    Rd = _rows_d(A)
    return C_BIAS + E + c * A + sum(((D >> (8 * j)) & 0xFF) * Rd[j] for j in range(72))


def tc_fold_cases_d(D, c, A):
    """(limb 0 of the assembled value below its top limb T, carry out of limb 8 in the
    fold, value >= m after the folds) for operand rows holding D and c."""
    v = tc_assembled_d(D, c, A)
    T, lo = v >> 576, v % B576
    add = T * ((1 << 240) - 1)
    past8 = (lo % B288) + add >= B288
    f = lo + add
    if f >= B576:
        f = f - B576 + (1 << 240) - 1
    return (lo & 0xFFFFFFFF) < T, past8, f >= M


def _canonical_state(D, c):
    """The LCG state X whose RANLUX form is (D, c), or None if (D, c) is not one."""
    X = R.to_lcg(D, c)
    if not 0 < X < M:
        return None
    return X if tuple(R.to_ranlux(X)) == (D, c) else None


def tc_d_borrow_states(A, rng: random.Random, want: int = 4):
    """States X whose RANLUX form (D, c) makes limb 0 of the assembled value smaller than
    16128 (so below the top limb, which is at least that), so that the fold borrows out of
    limb 0.  Limb 0 is sum_j d_j (R'_j mod 2^32) + c A + C + E mod 2^32; bytes 0..2 of D are
    searched over all 2^24 values for each random rest (about 63 qualify)."""
    import numpy as np
    Rd = _rows_d(A)
    E = (-C_BIAS) % M
    r = [x & 0xFFFFFFFF for x in Rd[:3]]
    grid = np.arange(1 << 24, dtype=np.uint64)
    part = (((grid & np.uint64(0xFF)) * np.uint64(r[0]) + ((grid >> np.uint64(8)) & np.uint64(0xFF)) * np.uint64(r[1])
             + (grid >> np.uint64(16)) * np.uint64(r[2])) & np.uint64(0xFFFFFFFF))
    found = []
    while len(found) < want:
        rest = rng.randrange(B576) & ~((1 << 24) - 1)
        c = rng.randrange(2)
        base = (C_BIAS + E + c * A + sum(((rest >> (8 * j)) & 0xFF) * Rd[j] for j in range(3, 72))) & 0xFFFFFFFF
        hits = np.nonzero(((part + np.uint64(base)) & np.uint64(0xFFFFFFFF)) < np.uint64(16128))[0]
        for h in hits[:8]:
            X = _canonical_state(rest | int(h), c)
            if X is not None and tc_fold_cases_d(rest | int(h), c, A)[0]:
                found.append(X)
                break
    return found


def tc_d_limb8_carry_states(A, rng: random.Random, want: int = 3):
    """States X whose RANLUX form (D, c) makes the fold carry out of limb 8, found as
    tc_limb8_carry_inputs finds operands: meeting in the middle over the low six bytes of
    D, for a random rest and borrow."""
    Rd = _rows_d(A)
    E = (-C_BIAS) % M
    width = 16128 << 240
    found = []
    while len(found) < want:
        base = rng.randrange(B576) & ~((1 << 48) - 1)
        c = rng.randrange(2)
        v0 = C_BIAS + E + c * A + sum(((base >> (8 * j)) & 0xFF) * Rd[j] for j in range(72))

        def side(j0):
            return [((a * Rd[j0] + b * Rd[j0 + 1] + cc * Rd[j0 + 2]) % B288, (a, b, cc))
                    for a in range(256) for b in range(256) for cc in range(4)]

        right = sorted(side(3))
        keys = [t[0] for t in right]
        for d_val, ta in side(0):
            a_val = (v0 + d_val) % B288
            lo = (B288 - width - a_val) % B288
            hi = (B288 - a_val) % B288
            spans = [(lo, hi)] if lo < hi else [(lo, B288), (0, hi)]
            hit = None
            for s, e in spans:
                for idx in range(bisect.bisect_left(keys, s), bisect.bisect_left(keys, e)):
                    tb = right[idx][1]
                    D = base | ta[0] | ta[1] << 8 | ta[2] << 16 | tb[0] << 24 | tb[1] << 32 | tb[2] << 40
                    if tc_fold_cases_d(D, c, A)[1]:
                        X = _canonical_state(D, c)
                        if X is not None:
                            hit = X
                            break
                if hit is not None:
                    break
            if hit is not None:
                found.append(hit)
                break
    return found


def tc_d_above_m_states(A, rs=(0, 1, 2, 5, 1 << 100, (1 << 239) + 7, (1 << 240) - 3)):
    """States X = A^-1 r mod m (product r below 2^240 - 1) whose operand rows (D, c) leave
    the folded value at r + m, which needs the final correction."""
    Ainv = pow(A, -1, M)
    out = []
    for r in rs:
        X = Ainv * r % M
        if 0 < X < M:
            D, c = R.to_ranlux(X)
            if tc_fold_cases_d(D, c, A)[2]:
                out.append(X)
    return out
