"""The CPU oracle against its pins (see oracle_pins.py for what each pin checks)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.fixture(scope="module", params=["default", "wide"])
def O(request):
    """Both builds of the oracle: widths 1-2, and the wide one (widths 1-4, pinned on 188- and 252-bit
    primes as well)."""
    return oracle.default() if request.param == "default" else oracle.wide()


@pytest.mark.parametrize("pin", oracle_pins.PINS, ids=[p.__name__ for p in oracle_pins.PINS])
def test_pin(O, pin):
    pin(O)
