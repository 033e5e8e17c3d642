"""Writes tests/golden/seed_vectors.txt from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py

The file freezes the oracle's first outputs for a few seeds and luxury levels, so that a
later change to the oracle's arithmetic shows up as a diff.  Its values come from
``oracle/ranluxpp.py`` alone; nothing here calls the CUDA library.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ranluxpp as R  # noqa: E402

SEEDS = (1, 2, 2718)          # 2718: the seed of the BigCrush run (Sec. 2.5)
LUXURY = (24, 223, 389, 2048)
N_U24 = 30                    # crosses one block boundary (24 words per block)
N_F64 = 15                    # crosses one block boundary (12 doubles per block)


def main():
    lines = ["# p seed kind index value_hex  (written by tests/golden/make_golden.py)"]
    for p in LUXURY:
        for s in SEEDS:
            u = R.Stream(p, seed=s).draw_u24(N_U24)
            for k, v in enumerate(u):
                lines.append(f"{p} {s} u24 {k} {v:06x}")
            f = R.Stream(p, seed=s).draw_f64(N_F64)
            for k, v in enumerate(f):
                lines.append(f"{p} {s} f64 {k} {R.f64_bits(v):016x}")
    path = os.path.join(ROOT, "tests", "golden", "seed_vectors.txt")
    with open(path, "w") as fh:
        fh.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
