"""Stored expected values (tests/golden/): the hand-worked fixtures parse and
agree with the definition in integer arithmetic, and the oracle still writes
the seeded fixture's values bit for bit (its arithmetic has not changed since
they were written)."""
import numpy as np

import golden
import synth
from golden import make_oracle_seeded as mk


def test_hand_worked_fixture_is_consistent():
    for c in golden.hand_worked():
        A = c["A"].astype(np.int64)
        B = c["B"].astype(np.int64)
        assert np.array_equal(A @ B, c["C"].astype(np.int64)), c["name"]
        assert np.array_equal(np.abs(A) @ np.abs(B), c["ABS"].astype(np.int64)), c["name"]


def test_seeded_fixture_inputs_are_the_generators():
    cases = {c["name"]: c for c in golden.oracle_seeded()}
    assert sorted(cases) == sorted(x[0] for x in mk.CASES)
    for name, n, m, p, gen, sa, sb in mk.CASES:
        c = cases[name]
        assert np.array_equal(c["A"], getattr(synth, gen)(sa, (n, m)))
        assert np.array_equal(c["B"], getattr(synth, gen)(sb, (m, p)))


def test_oracle_reproduces_seeded_fixture(orc):
    for c in golden.oracle_seeded():
        C, S = orc.gemm(c["A"], c["B"], with_abs=True)
        assert np.array_equal(C, c["C"]), c["name"]
        assert np.array_equal(S, c["ABS"]), c["name"]
