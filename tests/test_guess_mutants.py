"""Plant plausible mistakes in copies of the oracle's initial parameter
values (oracle/guess.py, Sec. 2.1.9) and check that the pins catch every one.

Each mutant is a one-expression edit of the module's source (a dropped clip,
swapped axes, a wrong sign, a wrong constant), loaded as a separate module."""
import importlib.util
import os

import pytest

from oracle import guess
from guess_pins import ALL_GUESS_PINS

SRC = guess.__file__

MUTANTS = [
    ("negative_light_counted", "I = np.maximum(np.asarray(cont, dtype=np.float64), 0.0)",
     "I = np.asarray(cont, dtype=np.float64)"),
    ("centroid_axes_swapped", "return float((I * x).sum() / s), float((I * y).sum() / s), float(s)",
     "return float((I * y).sum() / s), float((I * x).sum() / s), float(s)"),
    ("empty_map_centre_off_by_half", "return 0.5 * (nx - 1), 0.5 * (ny - 1), 0.0", "return 0.5 * nx, 0.5 * ny, 0.0"),
    ("moments_about_the_origin", "dx, dy = x - x0, y - y0", "dx, dy = x, y"),
    ("psf_variance_added", "lmax, lmin = lmax - v2, lmin - v2", "lmax, lmin = lmax + v2, lmin + v2"),
    ("axis_ratio_inverted", "c = math.sqrt(min(lmin / lmax, 1.0))", "c = math.sqrt(min(lmax / lmin, 1.0))"),
    ("axis_ratio_not_square_rooted", "c = math.sqrt(min(lmin / lmax, 1.0))", "c = min(lmin / lmax, 1.0)"),
    ("arcsin_for_arccos", "math.degrees(math.acos(c))", "math.degrees(math.asin(c))"),
    ("vsys_from_every_pixel", "use = near if near.any() else m", "use = m"),
    ("pa_halves_swapped", "d = a_v / a_c - b_v / b_c", "d = b_v / b_c - a_v / a_c"),
    ("pa_quarter_turn", "bins = (pa + np.arange(180)) % 360", "bins = (pa + 90 + np.arange(180)) % 360"),
    ("pa_polar_angle_in_radians", "phi = np.degrees(np.arctan2(dy[keep], dx[keep])) % 360.0",
     "phi = np.arctan2(dy[keep], dx[keep]) % 360.0"),
    ("pa_atan2_arguments_swapped", "phi = np.degrees(np.arctan2(dy[keep], dx[keep])) % 360.0",
     "phi = np.degrees(np.arctan2(dx[keep], dy[keep])) % 360.0"),
    ("rt_not_the_scale_length", "p[RT] = float(fixed[H])", "p[RT] = float(fixed[RT])"),
    ("epinat_slope_kept", "p[I0] = p[H] = 1.0", "p[I0] = 1.0"),
    ("start_velocities_swapped", "VT0, SIG0 = 150.0, 30.0", "VT0, SIG0 = 30.0, 150.0"),
]


def _load(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = os.path.join(str(tmp_path), "guess_%s.py" % name)
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))
    spec = importlib.util.spec_from_file_location("guess_" + name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(name, old, new, tmp_path):
    mod = _load(name, old, new, tmp_path)
    caught = []
    for pin in ALL_GUESS_PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, ZeroDivisionError, IndexError):
            caught.append(pin.__name__)
    assert caught, "no pin catches the mutant %s" % name


@pytest.mark.parametrize("pin", ALL_GUESS_PINS, ids=[p.__name__ for p in ALL_GUESS_PINS])
def test_the_unmutated_copy_passes(pin, tmp_path):
    pin(_load("identity", "import math", "import math", tmp_path))
