"""The integer-pipe elementary functions under the distribution draws (GPU).

-ln(w 2^-48), cos and sin of 2 pi v 2^-48 and the Box-Muller pair, each through its
C-ABI test entry point, against values computed here to 40 digits with Python's
decimal module (series written out below), and against CUDA's own double log, cos and
sin (through torch) within their stated bounds.  Inputs: crafted corners (powers of two,
the reduction-table interval edges, quarter turns, the extremes of the range) and seeded
random values."""
import math
import random
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

getcontext().prec = 50
TWO48 = 1 << 48


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_02504_gb300 as P
    return P.native


def run(fn, rows, per_out):
    x = torch.from_numpy(np.array(rows, dtype=np.uint64).reshape(-1).view(np.int64)).cuda()
    n = len(rows)
    out = torch.zeros(n * per_out, dtype=torch.int64, device="cuda")
    fn(x, out, n)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.float64).reshape(n, per_out)


def dec_pi():
    """pi by the Gauss-Legendre (arithmetic-geometric mean) iteration."""
    a, b, t, p = Decimal(1), Decimal(1) / Decimal(2).sqrt(), Decimal(1) / 4, Decimal(1)
    for _ in range(8):
        an = (a + b) / 2
        b = (a * b).sqrt()
        t -= p * (a - an) ** 2
        a, p = an, 2 * p
    return (a + b) ** 2 / (4 * t)


PI = dec_pi()


def dec_cos_sin_turns(v):
    """cos and sin of 2 pi v 2^-48: the angle folded to [-pi/4, pi/4] by whole quarter
    turns (exact in v), then the two Taylor series."""
    q = (v + (1 << 45)) >> 46                       # nearest quarter turn
    f = Decimal(v - (q << 46)) / Decimal(1 << 46)   # in [-1/2, 1/2) quarter turns
    th = f * PI / 2
    c, s, term, n = Decimal(0), Decimal(0), Decimal(1), 0
    while n < 60:
        if n % 4 == 0:
            c += term
        elif n % 4 == 1:
            s += term
        elif n % 4 == 2:
            c -= term
        else:
            s -= term
        n += 1
        term = term * th / n
    return [(c, s), (-s, c), (-c, -s), (s, -c)][q % 4]


def ulp(x):
    return math.ulp(abs(x)) if x else 0.0


def neg_ln_inputs():
    ws = {1, 2, 3, TWO48, TWO48 - 1, TWO48 - 2, TWO48 // 2, TWO48 // 2 + 1, 3 << 46}
    for k in range(49):
        for d in (-1, 0, 1):
            if 1 <= (1 << k) + d <= TWO48:
                ws.add((1 << k) + d)
    for kk in (1, 13, 30, 47, 48):           # the edges of every reduction interval
        for i in range(192, 385):
            base = (i << kk) >> 8
            for d in (-1, 0, 1):
                if 1 <= base + d <= TWO48:
                    ws.add(base + d)
    rng = random.Random(71)
    for _ in range(4000):
        ws.add(rng.randrange(1, TWO48 + 1))
        ws.add(max(1, int(2.0 ** rng.uniform(0, 48))))
        ws.add(TWO48 - rng.randrange(1, 1 << rng.randrange(1, 40)))
    return sorted(ws)


def test_neg_ln48_close_to_correctly_rounded(native):
    ws = neg_ln_inputs()
    got = run(native.rlxpp_test_neg_ln48, ws, 1)[:, 0]
    worst = 0.0
    for w, g in zip(ws, got):
        exact = -(Decimal(w) / TWO48).ln()
        err = abs(Decimal(g) - exact)
        # the fixed-point value is within 2^-60 x of -ln; rounding adds half an ulp
        assert err <= Decimal(ulp(float(exact))) / 2 + exact * Decimal(2.0 ** -60), (w, g, exact)
        if exact:
            worst = max(worst, float(err / Decimal(ulp(float(exact)))))
    assert worst <= 0.5 + 2 ** -6
    assert got[ws.index(TWO48)] == 0.0 and math.copysign(1, got[ws.index(TWO48)]) == 1.0
    assert got[ws.index(1)] == float(48 * Decimal(2).ln())


def test_neg_ln48_against_cuda_log(native):
    ws = neg_ln_inputs()
    got = run(native.rlxpp_test_neg_ln48, ws, 1)[:, 0]
    u = torch.tensor([w / TWO48 for w in ws], dtype=torch.float64, device="cuda")   # exact
    cuda = (-torch.log(u)).cpu().numpy()
    # CUDA's log is within 1 ulp; ours within half an ulp and a little
    tol = np.array([2 * ulp(c) for c in cuda])
    assert np.all(np.abs(got - cuda) <= tol)


def test_neg_ln48_rejects_out_of_range(native):
    got = run(native.rlxpp_test_neg_ln48, [0, TWO48 + 1, 2 ** 63], 1)[:, 0]
    assert np.all(np.isnan(got))


def cos_sin_inputs():
    vs = {0, 1, TWO48 - 1}
    for q in range(4):                          # quarter and eighth turns
        for d in (-1, 0, 1):
            vs.add(((q << 46) + d) % TWO48)
            vs.add(((q << 46) + (1 << 45) + d) % TWO48)
    for j in range(0, 257, 3):                  # table angles and the midpoints between them
        for d in (-1, 0, 1):
            vs.add(((j << 40) + d) % TWO48)
            vs.add(((j << 40) + (1 << 39) + d) % TWO48)
    rng = random.Random(72)
    for _ in range(3000):
        vs.add(rng.randrange(TWO48))
    return sorted(vs)


def test_cos_sin_2pi48(native):
    vs = cos_sin_inputs()
    got = run(native.rlxpp_test_cos_sin_2pi48, vs, 2)
    for v, (c, s) in zip(vs, got):
        ec, es = dec_cos_sin_turns(v)
        # the fixed-point values are within 2^-57; rounding to a double adds half an ulp
        for g, e in ((c, ec), (s, es)):
            assert abs(Decimal(g) - e) <= Decimal(ulp(float(e))) / 2 + Decimal(2.0 ** -57), (v, g, e)
        assert c * c + s * s == pytest.approx(1.0, abs=2 ** -50)
    # quarter turns are exact
    q = {v: (c, s) for v, (c, s) in zip(vs, got)}
    assert q[0] == (1.0, 0.0) and q[1 << 46] == (0.0, 1.0)
    assert q[2 << 46] == (-1.0, 0.0) and q[3 << 46] == (0.0, -1.0)
    # against CUDA's cos and sin of the double angle 2 pi d (itself rounded: about 2^-50)
    ang = torch.tensor([2 * math.pi * (v / TWO48) for v in vs], dtype=torch.float64, device="cuda")
    assert np.max(np.abs(got[:, 0] - torch.cos(ang).cpu().numpy())) < 2 ** -48
    assert np.max(np.abs(got[:, 1] - torch.sin(ang).cpu().numpy())) < 2 ** -48


def test_box_muller48(native):
    rng = random.Random(73)
    pairs = [(0, 0), (0, 1 << 46), (TWO48 - 1, 0), (TWO48 - 1, 1 << 45), (1, 3 << 46), (TWO48 // 2, 12345)]
    pairs += [(rng.randrange(TWO48), rng.randrange(TWO48)) for _ in range(3000)]
    pairs += [(TWO48 - rng.randrange(1, 1 << 20), rng.randrange(TWO48)) for _ in range(200)]
    pairs += [(rng.randrange(1, 1 << 20), rng.randrange(TWO48)) for _ in range(200)]
    got = run(native.rlxpp_test_box_muller48, pairs, 2)
    for (va, vb), (z0, z1) in zip(pairs, got):
        r = (-2 * (Decimal(TWO48 - va) / TWO48).ln()).sqrt()
        ec, es = dec_cos_sin_turns(vb)
        for z, e in ((z0, r * ec), (z1, r * es)):
            # r to 2^-58 relative (x to 2^-60), cos/sin to 2^-57, the final rounding half an ulp
            assert abs(Decimal(z) - e) <= Decimal(ulp(float(e))) / 2 + r * Decimal(2.0 ** -56), (va, vb, z, e)
    assert tuple(got[0]) == (0.0, 0.0)
    assert got[2][0] == pytest.approx(math.sqrt(96 * math.log(2)), rel=1e-15) and got[2][1] == 0.0
