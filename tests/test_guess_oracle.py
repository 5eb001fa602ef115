"""Pins of the oracle's initial parameter values (Sec. 2.1.9), on maps whose
answer the geometry fixes (the pins themselves are in tests/guess_pins.py,
shared with the mutant tests): point symmetry fixes the centroid and V_sys,
the field's antisymmetry about the minor axis fixes PA, and the second
moments of an exponential disc's elliptical isophotes fix cos^2 i (with the
PSF variance added to both axes when the map is convolved)."""
import pytest

from oracle import guess
from guess_pins import ALL_GUESS_PINS


@pytest.mark.parametrize("pin", ALL_GUESS_PINS, ids=[p.__name__ for p in ALL_GUESS_PINS])
def test_pin(pin):
    pin(guess)
