"""Stored expected values for the tests.

hand_worked.txt    products worked by hand from the paper's definition (cited
                   in the file).
oracle_seeded.txt  seeded inputs and the CPU oracle's FP64 results, written by
                   make_oracle_seeded.py, which calls only the oracle and the
                   seeded input generators.
"""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _parse(path, conv):
    cases = {}
    cur = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "n": int(tok[2]), "m": int(tok[3]), "p": int(tok[4])}
                cases[tok[1]] = cur
                continue
            cur.setdefault(tok[0], []).append([conv(t) for t in tok[1:]])
    out = []
    for c in cases.values():
        n, m, p = c["n"], c["m"], c["p"]
        rec = {"name": c["name"], "n": n, "m": m, "p": p}
        for key, shape, dt in (("A", (n, m), np.float32), ("B", (m, p), np.float32),
                               ("C", (n, p), np.float64), ("ABS", (n, p), np.float64)):
            if key in c:
                arr = np.array(c[key], dtype=np.float64)
                assert arr.shape == shape, (c["name"], key, arr.shape, shape)
                if dt is np.float32:
                    assert np.array_equal(arr.astype(np.float32).astype(np.float64), arr)
                rec[key] = arr.astype(dt)
        out.append(rec)
    return out


def hand_worked():
    """The hand-worked cases: list of dicts with n, m, p, A, B, C (and ABS)."""
    return _parse(os.path.join(HERE, "hand_worked.txt"), float)


def oracle_seeded():
    """The oracle-written seeded cases (hexadecimal floats, exact)."""
    return _parse(os.path.join(HERE, "oracle_seeded.txt"), float.fromhex)
