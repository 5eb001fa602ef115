"""The FP64 oracle against closed forms, invariants and brute force."""
import pytest

from oracle_pins import ALL_PINS


@pytest.mark.parametrize("pin", ALL_PINS, ids=[p.__name__ for p in ALL_PINS])
def test_pin(og, pin):
    pin(og)
