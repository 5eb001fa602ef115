"""Pins of the oracle's initial parameter values (Sec. 2.1.9), on maps whose
answer the geometry fixes: point symmetry fixes the centroid and V_sys, the
field's antisymmetry about the minor axis fixes PA, and the second moments
of an exponential disc's elliptical isophotes fix cos^2 i (with the PSF
variance added to both axes when the map is convolved)."""
import math

import numpy as np
import pytest

import oracle
from oracle import guess
from cases import ogeom
from paper_1510_01815_gb300.synth import Geometry, params as P


def _maps(g, p):
    m = oracle.evaluate(ogeom(g), p)
    return m[0], m[1], np.ones((g.ny, g.nx), np.uint8)


def test_centroid_and_vsys_of_a_point_symmetric_galaxy():
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    p = P(20.0, 20.0, 37.0, 55.0, 12.5, 180.0, 3.0, 40.0, 1.0, 4.0)
    cont, v, mask = _maps(g, p)
    x0, y0, s = guess.centroid(cont)
    assert s > 0 and abs(x0 - 20.0) < 1e-9 and abs(y0 - 20.0) < 1e-9
    # v - V_sys is odd under the point reflection, and the disc of radius 3
    # about the centre is symmetric under it
    assert abs(guess.systemic_velocity(v, mask, x0, y0) - 12.5) < 1e-9


@pytest.mark.parametrize("pa", [0.0, 37.0, 90.0, 200.0, 321.0])
def test_position_angle_of_a_rotating_disc(pa):
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    p = P(20.0, 20.0, pa, 50.0, 0.0, 180.0, 3.0, 40.0, 1.0, 4.0)
    _, v, mask = _maps(g, p)
    got = guess.position_angle(v, mask, 20.0, 20.0)
    d = abs((got - pa + 180.0) % 360.0 - 180.0)
    assert d <= 2.0, (pa, got)


@pytest.mark.parametrize("incl", [25.0, 45.0, 65.0])
def test_inclination_from_unconvolved_moments(incl):
    # h = 3 px in a 81 x 81 map: the disc is untruncated to e^-13
    g = Geometry(81, 81, 16, 50.0, 0.0, 0.0, 0.0)
    p = P(40.0, 40.0, 30.0, incl, 0.0, 100.0, 3.0, 40.0, 1.0, 3.0)
    cont, _, _ = _maps(g, p)
    assert abs(guess.photometric_inclination(cont, 40.0, 40.0, 0.0) - incl) < 0.6


@pytest.mark.parametrize("incl", [30.0, 60.0])
def test_inclination_corrects_the_psf_variance(incl):
    g = Geometry(81, 81, 16, 50.0, 0.0, 4.0, 0.0)
    sig = 4.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    p = P(40.0, 40.0, 120.0, incl, 0.0, 100.0, 3.0, 40.0, 1.0, 3.0)
    cont, _, _ = _maps(g, p)
    got = guess.photometric_inclination(cont, 40.0, 40.0, sig)
    assert abs(got - incl) < 0.5, got
    # leaving the correction out rounds the isophotes and biases i low
    assert guess.photometric_inclination(cont, 40.0, 40.0, 0.0) < incl - 1.0


def test_initial_guess_vector_and_degenerate_maps():
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    truth = P(20.0, 20.0, 200.0, 60.0, -7.0, 220.0, 2.0, 35.0, 1.0, 5.0)
    cont, v, mask = _maps(g, truth)
    sig = 2.5 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    q = guess.initial_guess(cont, v, mask, truth, sig)
    assert abs(q[0] - 20.0) < 1e-9 and abs(q[1] - 20.0) < 1e-9 and abs(q[4] + 7.0) < 1e-9
    assert abs((q[2] - 200.0 + 180.0) % 360.0 - 180.0) <= 2.0
    assert abs(q[3] - 60.0) < 4.0
    assert q[5] == guess.VT0 and q[7] == guess.SIG0 and q[6] == truth[9] and q[8] == truth[8] and q[9] == truth[9]
    # no light: the image centre; no usable velocity: V_sys 0 and PA 0
    z = np.zeros((9, 7))
    assert guess.centroid(z)[:2] == (3.0, 4.0)
    assert guess.systemic_velocity(z, np.zeros((9, 7), np.uint8), 3.0, 4.0) == 0.0
    assert guess.position_angle(z, np.zeros((9, 7), np.uint8), 3.0, 4.0) == 0.0
