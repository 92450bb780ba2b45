"""Every planted mistake in the oracle (a dropped term, a reversed index, a
sign error, a transposed operand, a missing reset, a normaliser without
absolute values, a Dot2 without compensation, a wrong sign in the complex
product) must fail at least one pin."""
import pytest

import oracle
from oracle import build as obuild
import oracle_pins

MUTANTS = list(range(1, 10))
MUTANTS.remove(6)  # 6 is unused (its slot was merged into 4)


@pytest.mark.parametrize("k", MUTANTS)
def test_mutant_is_caught(tmp_path, k):
    lib = obuild.build_mutant(k, str(tmp_path))
    orc = oracle.load(lib)
    assert orc.mutant() == k
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, "mutant %d passed every pin" % k
