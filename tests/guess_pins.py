"""Pins of the initial parameter values (Sec. 2.1.9) as functions of the
module under test, so that the same pins check oracle/guess.py and the
mutants planted in copies of it.  Each raises AssertionError when violated.

What fixes each answer: point symmetry fixes the centroid and V_sys; the
velocity field's antisymmetry about the minor axis fixes PA; an exponential
disc's elliptical isophotes give cos^2 i as the ratio of its second-moment
eigenvalues, with the PSF variance added to both when the map is convolved;
an untruncated disc's centroid is its centre wherever it sits."""
import math

import numpy as np

import oracle
from cases import ogeom
from paper_1510_01815_gb300.synth import Geometry, params as P


def _maps(g, p):
    m = oracle.evaluate(ogeom(g), p)
    return m[0], m[1], np.ones((g.ny, g.nx), np.uint8)


def pin_centroid_and_vsys_of_a_point_symmetric_galaxy(guess):
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    p = P(20.0, 20.0, 37.0, 55.0, 12.5, 180.0, 3.0, 40.0, 1.0, 4.0)
    cont, v, mask = _maps(g, p)
    x0, y0, s = guess.centroid(cont)
    assert s > 0 and abs(x0 - 20.0) < 1e-9 and abs(y0 - 20.0) < 1e-9
    # v - V_sys is odd under the point reflection, and the disc of radius 2.5
    # about the centre is symmetric under it
    assert abs(guess.systemic_velocity(v, mask, x0, y0) - 12.5) < 1e-9


def pin_centroid_of_an_off_centre_disc(guess):
    # h = 2.5 px, centre (31.3, 48.6) in a 81 x 96 map: the disc is
    # untruncated to e^-12, so its centroid is its centre (x and y differ)
    g = Geometry(81, 96, 8, 50.0, 0.0, 0.0, 0.0)
    p = P(31.3, 48.6, 30.0, 50.0, 0.0, 20.0, 3.0, 40.0, 1.0, 2.5)  # lines far inside the band
    cont, _, _ = _maps(g, p)
    x0, y0, _ = guess.centroid(cont)
    assert abs(x0 - 31.3) < 1e-3 and abs(y0 - 48.6) < 1e-3, (x0, y0)


def pin_negative_continuum_values_count_as_zero(guess):
    g = Geometry(41, 41, 16, 20.0, 0.0, 2.5, 30.0)
    p = P(20.0, 20.0, 37.0, 55.0, 0.0, 180.0, 3.0, 40.0, 1.0, 4.0)
    cont, _, _ = _maps(g, p)
    zero, blem = cont.copy(), cont.copy()
    zero[3, 35] = 0.0
    blem[3, 35] = -5.0 * cont.max()  # a negative artefact far from the centre
    a, b = guess.centroid(zero), guess.centroid(blem)
    assert a == b
    ia = guess.photometric_inclination(zero, a[0], a[1], 0.0)
    assert guess.photometric_inclination(blem, a[0], a[1], 0.0) == ia


def pin_vsys_is_taken_near_the_centre(guess):
    # the receding outer half masked away: the mean of all unmasked pixels is
    # biased low, the mean within 2.5 px of the centre is still V_sys
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    p = P(20.0, 20.0, 90.0, 55.0, 7.0, 180.0, 3.0, 40.0, 1.0, 4.0)
    _, v, mask = _maps(g, p)
    y, x = np.mgrid[0:41, 0:41]
    mask = mask.copy()
    mask[(v > 7.0) & ((x - 20.0) ** 2 + (y - 20.0) ** 2 > 16.0)] = 0
    assert abs(float(v[mask != 0].mean()) - 7.0) > 5.0  # the global mean is biased
    assert abs(guess.systemic_velocity(v, mask, 20.0, 20.0) - 7.0) < 1e-9


def pin_position_angle_of_a_rotating_disc(guess):
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    for pa in (0.0, 37.0, 90.0, 200.0, 321.0):
        p = P(20.0, 20.0, pa, 50.0, 0.0, 180.0, 3.0, 40.0, 1.0, 4.0)
        _, v, mask = _maps(g, p)
        got = guess.position_angle(v, mask, 20.0, 20.0)
        assert abs((got - pa + 180.0) % 360.0 - 180.0) <= 2.0, (pa, got)


def pin_inclination_from_unconvolved_moments(guess):
    # h = 3 px in a 81 x 81 map: the disc is untruncated to e^-13
    g = Geometry(81, 81, 16, 50.0, 0.0, 0.0, 0.0)
    for incl in (25.0, 45.0, 65.0):
        p = P(40.0, 40.0, 30.0, incl, 0.0, 100.0, 3.0, 40.0, 1.0, 3.0)
        cont, _, _ = _maps(g, p)
        assert abs(guess.photometric_inclination(cont, 40.0, 40.0, 0.0) - incl) < 0.6, incl


def pin_inclination_corrects_the_psf_variance(guess):
    g = Geometry(81, 81, 16, 50.0, 0.0, 4.0, 0.0)
    sig = 4.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    for incl in (30.0, 60.0):
        p = P(40.0, 40.0, 120.0, incl, 0.0, 100.0, 3.0, 40.0, 1.0, 3.0)
        cont, _, _ = _maps(g, p)
        got = guess.photometric_inclination(cont, 40.0, 40.0, sig)
        assert abs(got - incl) < 0.5, (incl, got)
        # leaving the correction out rounds the isophotes and biases i low
        assert guess.photometric_inclination(cont, 40.0, 40.0, 0.0) < incl - 1.0


def pin_initial_guess_vector_and_degenerate_maps(guess):
    g = Geometry(41, 41, 64, 20.0, 0.0, 2.5, 30.0)
    truth = P(20.0, 20.0, 200.0, 60.0, -7.0, 220.0, 2.0, 35.0, 1.0, 5.0)
    cont, v, mask = _maps(g, truth)
    sig = 2.5 / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    q = guess.initial_guess(cont, v, mask, truth, sig)
    assert abs(q[0] - 20.0) < 1e-9 and abs(q[1] - 20.0) < 1e-9 and abs(q[4] + 7.0) < 1e-9
    assert abs((q[2] - 200.0 + 180.0) % 360.0 - 180.0) <= 2.0
    assert abs(q[3] - 60.0) < 4.0
    assert q[5] == 150.0 and q[7] == 30.0 and q[6] == truth[9] and q[8] == truth[8] and q[9] == truth[9]
    # velocity fields: r_t is the caller's, the Epinat slopes start at 1
    f = truth.copy()
    f[6] = 3.3
    qv = guess.initial_guess(cont, v, mask, f, sig, model=2)
    assert qv[6] == 3.3 and qv[8] == 1.0 and qv[9] == 1.0
    # no light: the image centre; no usable velocity: V_sys 0 and PA 0
    z = np.zeros((9, 7))
    assert guess.centroid(z)[:2] == (3.0, 4.0)
    assert guess.systemic_velocity(z, np.zeros((9, 7), np.uint8), 3.0, 4.0) == 0.0
    assert guess.position_angle(z, np.zeros((9, 7), np.uint8), 3.0, 4.0) == 0.0


ALL_GUESS_PINS = [
    pin_centroid_and_vsys_of_a_point_symmetric_galaxy,
    pin_centroid_of_an_off_centre_disc,
    pin_negative_continuum_values_count_as_zero,
    pin_vsys_is_taken_near_the_centre,
    pin_position_angle_of_a_rotating_disc,
    pin_inclination_from_unconvolved_moments,
    pin_inclination_corrects_the_psf_variance,
    pin_initial_guess_vector_and_degenerate_maps,
]
