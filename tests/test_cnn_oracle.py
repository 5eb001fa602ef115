"""Pins of the CNN oracle (oracle/cnn.py); the pins are in tests/cnn_pins.py,
shared with the mutant tests."""
import pytest

from oracle import cnn
from cnn_pins import ALL_CNN_PINS


@pytest.mark.parametrize("pin", ALL_CNN_PINS, ids=[p.__name__ for p in ALL_CNN_PINS])
def test_pin(pin):
    pin(cnn)
