"""Seeded synthetic inputs for the disc-galaxy workloads.

This module only draws numbers: parameter sets, noise, masks and cube shapes.
It holds none of the forward model's arithmetic, so both the CUDA path and the
FP64 oracle can consume what it produces.  Every draw goes through
``numpy.random.default_rng(seed)``.

The shapes and ranges stand in for the paper's mock data (Sec. 3.1, Table 2),
its Fabry-Perot survey (GHASP, Sec. 3.2) and its IFU survey (DYNAMO,
Sec. 3.3), whose data are not available here.
"""
from dataclasses import dataclass, asdict, replace

import numpy as np

NPAR = 10
X0, Y0, PA, INCL, VSYS, VMAX, RT, SIG0, I0, H = range(NPAR)
PARAM_NAMES = ("x0", "y0", "pa", "incl", "vsys", "vmax", "rt", "sig0", "i0", "h")

# Parameters the fits leave free: I0 and h are fixed (Sec. 2.1.6).
FREE_DEFAULT = (X0, Y0, PA, INCL, VSYS, VMAX, RT, SIG0)


@dataclass(frozen=True)
class Geometry:
    """Data cube nx x ny spaxels x nz channels of width dv (km/s) centred on
    vc; PSF FWHM in pixels; LSF FWHM in km/s; LSF mode 0 (3-axis convolution)
    or 1 (LSF folded into the line width); upsampling factor; kernel radius
    in sigmas."""
    nx: int
    ny: int
    nz: int
    dv: float
    vc: float = 0.0
    psf_fwhm: float = 0.0
    lsf_fwhm: float = 0.0
    lsf_mode: int = 0
    upsample: int = 1
    halo_sigmas: float = 4.0
    model: int = 0  # 0 intensity cube; 1 velocity field (arctan); 2 velocity field (Epinat)

    def asdict(self):
        return asdict(self)

    def with_(self, **kw):
        return replace(self, **kw)


def params(x0, y0, pa, incl, vsys, vmax, rt, sig0, i0, h):
    return np.array([x0, y0, pa, incl, vsys, vmax, rt, sig0, i0, h], dtype=np.float64)


# ----------------------------------------------------------------------------
# Single galaxy, plain LM fit: 32x32 spaxels x 64 channels at 20 km/s.
SINGLE_GEOM = Geometry(32, 32, 64, 20.0, 0.0, 2.5, 30.0)
SINGLE_TRUTH = params(15.5, 15.5, 120.0, 55.0, 0.0, 200.0, 3.0, 40.0, 1.0, 4.0)
SINGLE_NOISE_V = 5.0

# Fabry-Perot-like galaxy: 192x192 x 48 channels at 10 km/s (GHASP-like
# seeing of 3 px and spectral resolution of 30 km/s).
FP_GEOM = Geometry(192, 192, 48, 10.0, 0.0, 3.0, 30.0)
FP_RANGES = {PA: (0.0, 360.0), INCL: (20.0, 80.0), VMAX: (50.0, 300.0),
             RT: (1.0, 8.0), SIG0: (10.0, 80.0)}
FP_SCALE_LENGTH = 20.0
FP_LIVE_POINTS = 400

# Nested-grid brute force: 64x64 x 64 channels.
GRID_GEOM = Geometry(64, 64, 64, 20.0, 0.0, 2.5, 30.0)

# Learned-seed training data: 64x64 maps from 64-channel cubes.
CNN_GEOM = Geometry(64, 64, 64, 20.0, 0.0, 2.5, 30.0)


# CNN seed workload: 64 x 64 maps; Table 2-like ranges extended to the
# Fabry-Perot ones, centre within 0.4-0.6 of the frame, I0 = 1.
CNN_RANGES = {X0: (25.6, 38.4), Y0: (25.6, 38.4), PA: (0.0, 360.0), INCL: (20.0, 80.0), VSYS: (-30.0, 30.0),
              VMAX: (50.0, 300.0), RT: (1.0, 8.0), SIG0: (10.0, 80.0), H: (4.0, 10.0)}


def draw_cnn_params(rng, n):
    p = np.zeros((n, NPAR))
    for k, (lo, hi) in CNN_RANGES.items():
        p[:, k] = rng.uniform(lo, hi, n)
    p[:, I0] = 1.0
    return p


def draw_fp_params(rng, n, geom=FP_GEOM, h=FP_SCALE_LENGTH):
    """Parameter sets over the Fabry-Perot ranges; x0, y0 in 0.4-0.6 N."""
    p = np.zeros((n, NPAR))
    p[:, X0] = rng.uniform(0.4 * geom.nx, 0.6 * geom.nx, n)
    p[:, Y0] = rng.uniform(0.4 * geom.ny, 0.6 * geom.ny, n)
    for k, (lo, hi) in FP_RANGES.items():
        p[:, k] = rng.uniform(lo, hi, n)
    p[:, VSYS] = 0.0
    p[:, I0] = 1.0
    p[:, H] = h
    return p


def fp_prior_box(geom=FP_GEOM, h=FP_SCALE_LENGTH):
    """Uniform prior box (lo, hi) over all ten parameters; fixed ones have
    lo == hi."""
    lo = np.zeros(NPAR)
    hi = np.zeros(NPAR)
    lo[X0], hi[X0] = 0.4 * geom.nx, 0.6 * geom.nx
    lo[Y0], hi[Y0] = 0.4 * geom.ny, 0.6 * geom.ny
    for k, (a, b) in FP_RANGES.items():
        lo[k], hi[k] = a, b
    lo[I0] = hi[I0] = 1.0
    lo[H] = hi[H] = h
    return lo, hi


def perturb(rng, p, free=FREE_DEFAULT, frac=0.2, lo=None, hi=None):
    """Start point: each free parameter scaled by 1 + U(-frac, frac); a
    parameter whose value is 0 is moved by U(-frac, frac) * scale instead
    (scale 20 km/s for Vsys).  Clipped to [lo, hi] when given."""
    q = np.array(p, dtype=np.float64, copy=True)
    for k in free:
        u = rng.uniform(-frac, frac)
        if q[k] == 0.0:
            q[k] = u * 20.0
        else:
            q[k] = q[k] * (1.0 + u)
    if lo is not None:
        q = np.minimum(np.maximum(q, lo), hi)
    return q


def gaussian_noise(rng, shape, sigma):
    return rng.normal(0.0, sigma, size=shape)


def dead_fibre_mask(rng, shape, frac=0.02):
    """1 = usable, 0 = dead fibre / detector pixel (Sec. 3.1)."""
    return (rng.uniform(size=shape) >= frac).astype(np.uint8)


def sn_mask(m0, threshold=3.0, eta=0.01):
    """S/N mask from a noiseless integrated-intensity map: S/N is m0 over a
    flux noise of eta * max(m0); spaxels below ``threshold`` are masked."""
    m0 = np.asarray(m0, dtype=np.float64)
    noise = eta * float(m0.max())
    return (m0 >= threshold * noise).astype(np.uint8)


def weights(shape, e_v, w_sigma=1.0):
    """w_v = 1/E_v; w_s = sqrt(W)/E_s with E_s = sqrt(2) E_v (Sec. 3.1)."""
    e_s = np.sqrt(2.0) * e_v
    return (np.full(shape, 1.0 / e_v, dtype=np.float32),
            np.full(shape, np.sqrt(w_sigma) / e_s, dtype=np.float32))


# ----------------------------------------------------------------------------
# Survey batch: uneven cubes, log-uniform 24-96 spatial and 32-128 channels,
# parameters from the mock parameter space (Table 2).
SURVEY_PSF_FWHM = 4.0


def draw_survey(rng, n, nxy_range=(24, 96)):
    """Returns a list of (Geometry, true params) for n survey galaxies
    (spatial size log-uniform over nxy_range; the mock dataset of Sec. 3.1
    uses 32 - 96)."""
    out = []
    for _ in range(n):
        nxy = int(round(np.exp(rng.uniform(np.log(nxy_range[0]), np.log(nxy_range[1])))))
        nz = int(round(np.exp(rng.uniform(np.log(32), np.log(128)))))
        pa = rng.uniform(0.0, 45.0)
        incl = rng.uniform(5.0, 85.0)
        rt = rng.uniform(0.5, 2.0) * SURVEY_PSF_FWHM
        h = rng.uniform(1.0, 3.0) * SURVEY_PSF_FWHM
        vt = rng.uniform(50.0, 300.0)
        sig = rng.uniform(20.0, 100.0)
        lsf = rng.uniform(20.0, 60.0)
        x0 = rng.uniform(0.4 * nxy, 0.6 * nxy)
        y0 = rng.uniform(0.4 * nxy, 0.6 * nxy)
        # Channel width that keeps the whole line inside the band.
        s_line = np.hypot(sig, lsf / 2.3548200450309493)
        span = vt * np.sin(np.radians(incl)) + 4.0 * s_line
        dv = max(10.0, float(np.ceil(2.0 * span / nz)))
        g = Geometry(nxy, nxy, nz, dv, 0.0, SURVEY_PSF_FWHM, lsf)
        out.append((g, params(x0, y0, pa, incl, 0.0, vt, rt, sig, 1.0, h)))
    return out
