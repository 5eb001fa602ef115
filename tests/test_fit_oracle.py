"""Pins of the oracle's optimisers (oracle/fit.py: LM, nested grids, nested
sampling); the pins are in tests/fit_pins.py, shared with the mutant tests."""
import pytest

from oracle import fit
from fit_pins import ALL_FIT_PINS


@pytest.mark.parametrize("pin", ALL_FIT_PINS, ids=[p.__name__ for p in ALL_FIT_PINS])
def test_pin(pin):
    pin(fit)
