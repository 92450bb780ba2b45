"""The CPU oracle against its pins (runs without a GPU)."""
import pytest

import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    assert orc.mutant() == 0
    pin(orc)
