"""The oracle on the GPU machine's own host (an Arm CPU, where the CPU suite runs on
x86): the stored golden vectors, written on another machine by tests/golden/make_golden.py
from the oracle, must come out identically from the Python oracle and from the C
recurrence oracle built there (the method is integer arithmetic throughout, so the
sequences do not depend on the platform).  Marked gpu so that it runs on that machine;
it uses no GPU."""
import os

import numpy as np
import pytest

from oracle import ranluxpp as R
from oracle import swb_lib as S
from tests.oracle_side import StreamSet

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "seed_vectors.txt")


def _rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            p, s, kind, k, v = line.split()
            rows.append((int(p), int(s), kind, int(k), int(v, 16)))
    return rows


def test_golden_vectors_on_this_host():
    rows = _rows()
    assert rows
    by_key = {}
    for p, s, kind, k, v in rows:
        by_key.setdefault((p, s, kind), []).append((k, v))
    for (p, s, kind), kv in by_key.items():
        n = max(k for k, _ in kv) + 1
        st = R.Stream(p, seed=s)
        py = st.draw_u24(n) if kind == "u24" else [R.f64_bits(x) for x in st.draw_f64(n)]
        c = StreamSet.from_seeds([s], p).draw(n, S.KIND_U24 if kind == "u24" else S.KIND_F64)[0]
        c = c.view(np.uint32) if kind == "u24" else c.view(np.uint64)
        for k, v in kv:
            assert py[k] == v and int(c[k]) == v, (p, s, kind, k)
