"""Initial model parameter values (Sec. 2.1.9), FP64 (TEST INFRASTRUCTURE).

Only the tests, the smoke check and the benchmark's CPU legs may import this
module; the library computes the same quantities in its own kernel and
shares nothing with it.

The paper starts its optimisers from values measured on the observation's
continuum, velocity and dispersion maps.  Its description leaves details
open, which are read as follows:
  - centre (x0, y0): the intensity-weighted mean position of the continuum
    map (negative values count as 0);
  - V_sys: the mean of the velocity map over unmasked pixels within
    VSYS_RADIUS pixels of that centre (all unmasked pixels if none is that
    close);
  - PA: the line through the centre that splits the velocity field so that
    the difference of the two parts' means is largest.  With x_e =
    -dx sin PA + dy cos PA = r sin(phi - PA) (Eqs. 1-2, phi the polar angle
    of the pixel about the centre), the receding half x_e > 0 is the polar
    angle range (PA, PA + 180 deg); PA runs over whole degrees 0 .. 359, the
    pixels are binned by whole degrees of phi, and the largest
    mean(x_e > 0) - mean(x_e < 0) wins (ties to the smallest PA);
  - i: the paper takes a photometric inclination from a catalogue; here it
    is measured on the continuum map the same way: the eigenvalues of its
    intensity-weighted second central moments, less the PSF variance (the
    moments of a convolution with a Gaussian add), give cos^2 i as their
    ratio; i is clipped to [INCL_MIN, INCL_MAX];
  - r_t: the photometric scale radius: for the cube model the scale length
    h, which is known and fixed (as is I0); for a velocity field (no
    intensity model) the caller's value in the r_t slot;
  - V_t = 150 km/s, sigma0 = 30 km/s; for the Epinat curve a = g = 1.
"""
import math

import numpy as np

VSYS_RADIUS = 2.5  # no pixel of the grid lies at exactly this distance from a pixel centre
INCL_MIN, INCL_MAX = 5.0, 85.0
VT0, SIG0 = 150.0, 30.0
NPAR = 10
X0, Y0, PA, INCL, VSYS, VMAX, RT, SIG, I0, H = range(10)


def centroid(cont):
    """Intensity-weighted mean position (x, y) and the weights' sum."""
    I = np.maximum(np.asarray(cont, dtype=np.float64), 0.0)
    ny, nx = I.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = I.sum()
    if not s > 0:
        return 0.5 * (nx - 1), 0.5 * (ny - 1), 0.0
    return float((I * x).sum() / s), float((I * y).sum() / s), float(s)


def photometric_inclination(cont, x0, y0, psf_sigma):
    """Inclination (deg) from the continuum's second central moments about
    (x0, y0), each eigenvalue less the PSF variance."""
    I = np.maximum(np.asarray(cont, dtype=np.float64), 0.0)
    ny, nx = I.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    s = I.sum()
    if not s > 0:
        return 0.5 * (INCL_MIN + INCL_MAX)
    dx, dy = x - x0, y - y0
    mxx, myy, mxy = (I * dx * dx).sum() / s, (I * dy * dy).sum() / s, (I * dx * dy).sum() / s
    tr, det = mxx + myy, mxx * myy - mxy * mxy
    disc = math.sqrt(max(0.25 * tr * tr - det, 0.0))
    lmax, lmin = 0.5 * tr + disc, 0.5 * tr - disc
    v2 = psf_sigma * psf_sigma
    lmax, lmin = lmax - v2, lmin - v2
    if not (lmax > 0.0 and lmin > 0.0):
        return 0.5 * (INCL_MIN + INCL_MAX) if not lmax > 0.0 else INCL_MAX
    c = math.sqrt(min(lmin / lmax, 1.0))
    return float(min(max(math.degrees(math.acos(c)), INCL_MIN), INCL_MAX))


def systemic_velocity(v, mask, x0, y0):
    v = np.asarray(v, dtype=np.float64)
    m = np.asarray(mask) != 0
    ny, nx = v.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    near = m & ((x - x0) ** 2 + (y - y0) ** 2 <= VSYS_RADIUS ** 2)
    use = near if near.any() else m
    return float(v[use].mean()) if use.any() else 0.0


def position_angle(v, mask, x0, y0):
    """Whole-degree PA maximising mean(v | x_e > 0) - mean(v | x_e < 0)."""
    v = np.asarray(v, dtype=np.float64)
    m = np.asarray(mask) != 0
    ny, nx = v.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    dx, dy = x - x0, y - y0
    keep = m & ((dx != 0.0) | (dy != 0.0))
    phi = np.degrees(np.arctan2(dy[keep], dx[keep])) % 360.0
    b = np.minimum(np.floor(phi).astype(int), 359)
    sv = np.bincount(b, weights=v[keep], minlength=360)
    cn = np.bincount(b, minlength=360).astype(np.float64)
    best, best_d = 0, -np.inf
    tot_v, tot_c = sv.sum(), cn.sum()
    for pa in range(360):
        bins = (pa + np.arange(180)) % 360   # polar angles (pa, pa + 180)
        a_v, a_c = sv[bins].sum(), cn[bins].sum()
        b_v, b_c = tot_v - a_v, tot_c - a_c
        if a_c == 0 or b_c == 0:
            continue
        d = a_v / a_c - b_v / b_c
        if d > best_d:
            best, best_d = pa, d
    return float(best)


def initial_guess(cont, v, mask, fixed, psf_sigma, model=0):
    """Parameter vector of Sec. 2.1.9 for one galaxy; `fixed` supplies I0 and
    h (cube model, r_t := h) or r_t (velocity fields); the Epinat slopes, in
    the I0 and h slots of a velocity field, are set to 1."""
    p = np.array(fixed, dtype=np.float64, copy=True)
    x0, y0, _ = centroid(cont)
    p[X0], p[Y0] = x0, y0
    p[VSYS] = systemic_velocity(v, mask, x0, y0)
    p[PA] = position_angle(v, mask, x0, y0)
    p[INCL] = photometric_inclination(cont, x0, y0, psf_sigma)
    p[VMAX] = VT0
    p[SIG] = SIG0
    if model == 0:
        p[RT] = float(fixed[H])
    if model == 2:
        p[I0] = p[H] = 1.0
    return p
