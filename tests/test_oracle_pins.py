"""The CPU oracle against its pins (see oracle_pins.py for what each pin checks)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.fixture(scope="module")
def O():
    return oracle.default()


@pytest.mark.parametrize("pin", oracle_pins.PINS, ids=[p.__name__ for p in oracle_pins.PINS])
def test_pin(O, pin):
    pin(O)
