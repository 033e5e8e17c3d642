"""The constant tables of the integer-pipe elementary functions (host only).

The committed header must be exactly what its generator writes, and the entries are
checked against values computed independently here: ln 2 and pi/4 against their
published hexadecimal expansions, the reduction table's reciprocals against their
defining bounds, ln R and the first-quadrant sines and cosines against Python's math
within a few units of its double precision."""
import importlib.util
import math
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2106_02504_gb300", "csrc")


def load_generator():
    spec = importlib.util.spec_from_file_location("gen_fixmath_tables", os.path.join(CSRC, "gen_fixmath_tables.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def header():
    with open(os.path.join(CSRC, "rlxpp_fixmath_tables.h")) as f:
        return f.read()


def test_header_is_generated():
    assert load_generator().render() == header()


def parse():
    h = header()
    ln2 = int(re.search(r"kLn2Hi = 0x([0-9a-f]+)", h).group(1), 16) << 64
    ln2 |= int(re.search(r"kLn2Lo = 0x([0-9a-f]+)", h).group(1), 16)
    two_pi = int(re.search(r"kTwoPi61 = 0x([0-9a-f]+)", h).group(1), 16)
    rows = [(int(a, 16), int(b, 16)) for a, b in re.findall(r"\{0x([0-9a-f]+)ull, 0x([0-9a-f]+)ull\}", h)]
    return ln2, two_pi, rows[:384], rows[384:]


def rounded_shift(v, k):
    return (v + (1 << (k - 1))) >> k


def test_constants_match_published_expansions():
    ln2, two_pi, _, _ = parse()
    # ln 2 = 0.B17217F7D1CF79ABC9E3B39803F2F6AF40F3... (hexadecimal)
    assert ln2 == rounded_shift(0xB17217F7D1CF79ABC9E3B39803F2F6AF40F3, 4 * 36 - 120)
    # pi / 4 = 0.C90FDAA22168C234C4C6628B80DC1CD1... and 2 pi 2^61 = (pi / 4) 2^64
    assert two_pi == rounded_shift(0xC90FDAA22168C234C4C6628B80DC1CD1, 4 * 32 - 64)


def test_log_reduction_table():
    _, _, ln_rows, _ = parse()
    assert len(ln_rows) == 384
    for k, (lo, hi) in enumerate(ln_rows):
        i = 384 + k
        rint = lo & 0xFFFF
        # R = rint / 2^15 is the largest 16-bit value with m R <= 1 on (i/512, (i+1)/512]
        assert (i + 1) * rint <= 512 * 2 ** 15 < (i + 1) * (rint + 1)
        # and m R >= 1 - 2^-8.5 at the interval's lower end
        assert 1 - i * rint / (512 * 2 ** 15) <= 2 ** -8.5
        v = ((hi << 64) | (lo & ~0xFFFF))
        if v >= 1 << 127:
            v -= 1 << 128
        want = math.log(rint / 2 ** 15)
        assert abs(v / 2 ** 120 - want) <= 4 * math.ulp(abs(want)) + 2 ** -100, i
    assert ln_rows[511 - 384] == (1 << 15, 0)           # R = 1, ln R = 0 for (511/512, 1]


def test_sin_cos_table():
    _, _, _, sc = parse()
    assert len(sc) == 65
    assert sc[0] == (0, 1 << 63) and sc[64] == (1 << 63, 0)
    for j, (s, c) in enumerate(sc):
        a = 2 * math.pi * j / 256
        assert abs(s / 2 ** 63 - math.sin(a)) <= 2 ** -51 and abs(c / 2 ** 63 - math.cos(a)) <= 2 ** -51, j
        assert (s * s + c * c) / 2 ** 126 == __import__("pytest").approx(1.0, abs=2 ** -60)
        assert sc[64 - j] == (c, s)                      # sin and cos swap at a quarter turn
