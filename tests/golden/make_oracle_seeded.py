"""Writes oracle_seeded.txt: small seeded products and the CPU oracle's FP64
results (and |A||B| normalisers) as hexadecimal floats.  It calls only the
oracle and the seeded input generators.

  python tests/golden/make_oracle_seeded.py
"""
from __future__ import annotations

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

# (name, n, m, p, generator, seed of A, seed of B): shapes that are not
# multiples of any tile, a long inner dimension, and integer entries
CASES = [
    ("uniform_5x7x3", 5, 7, 3, "uniform_pm1", 2000, 2001),
    ("uniform_13x24x9", 13, 24, 9, "uniform_pm1", 2002, 2003),
    ("uniform_2x100x3", 2, 100, 3, "uniform_pm1", 2004, 2005),
    ("small_ints_9x33x11", 9, 33, 11, "small_ints", 2006, 2007),
]


def main() -> int:
    orc = oracle.default()
    lines = ["# Seeded inputs (synth.<generator>(seed, shape)) and the CPU oracle's FP64",
             "# product C and normaliser ABS = |A||B|, hexadecimal floats.",
             "# Written by make_oracle_seeded.py (calls only the oracle).",
             "# Format: case <name> <n> <m> <p>, then A, B, C and ABS rows."]
    for name, n, m, p, gen, sa, sb in CASES:
        A = getattr(synth, gen)(sa, (n, m))
        B = getattr(synth, gen)(sb, (m, p))
        C, S = orc.gemm(A, B, with_abs=True)
        lines.append("# %s: synth.%s(%d, (%d, %d)), synth.%s(%d, (%d, %d))" % (
            name, gen, sa, n, m, gen, sb, m, p))
        lines.append("case %s %d %d %d" % (name, n, m, p))
        for key, X in (("A", A), ("B", B), ("C", C), ("ABS", S)):
            for row in X:
                lines.append(key + " " + " ".join(float(v).hex() for v in row))
    with open(os.path.join(HERE, "oracle_seeded.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("wrote", os.path.join(HERE, "oracle_seeded.txt"))
    return 0


if __name__ == "__main__":
    sys.exit(main())
