"""The CPU oracle against facts outside itself (see tests/pins.py)."""
import pytest

from pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_pin_holds(pin):
    failures = pin()
    assert not failures, failures
