"""FP64 CPU oracle of the disc-galaxy forward model (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the arithmetic lives in ``gbk_oracle.c`` (plain C, FP64) and this
module only marshals numpy arrays to it.  The fitting algorithms built on it
(Levenberg-Marquardt, nested grids, nested sampling) are in ``oracle.fit``.

Paper: Bekiaris et al. 2015, "Kinematic modelling of disc galaxies using
graphics processing units" (arXiv:1510.01815).  Each C function cites the
section and equation it follows.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

NPAR = 10
X0, Y0, PA, INCL, VSYS, VMAX, RT, SIG0, I0, H = range(NPAR)
PARAM_NAMES = ("x0", "y0", "pa", "incl", "vsys", "vmax", "rt", "sig0", "i0", "h")
FWHM_PER_SIGMA = 2.3548200450309493


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("upsample", ctypes.c_int32), ("dv", ctypes.c_double), ("vc", ctypes.c_double),
                ("psf_fwhm", ctypes.c_double), ("lsf_fwhm", ctypes.c_double),
                ("lsf_mode", ctypes.c_int32), ("model", ctypes.c_int32),
                ("halo_sigmas", ctypes.c_double)]


@dataclass(frozen=True)
class Geom:
    """Observation geometry: data cube nx x ny x nz, channel width dv (km/s),
    band centre vc, PSF FWHM (pixels), LSF FWHM (km/s), LSF mode (0: z
    convolution, 1: folded into the line width), upsampling u, kernel
    truncation radius in sigmas."""
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

    def c(self):
        return _Geom(self.nx, self.ny, self.nz, self.upsample, self.dv, self.vc,
                     self.psf_fwhm, self.lsf_fwhm, self.lsf_mode, self.model, self.halo_sigmas)


_lib = None


def lib():
    if _lib is None:
        use_library(_build.build())
    return _lib


def use_library(path):
    """Load the oracle from ``path`` (the tests use this to load deliberately
    broken copies and check that the pins catch them)."""
    global _lib
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    up = ctypes.POINTER(ctypes.c_uint8)
    ip = ctypes.POINTER(ctypes.c_int32)
    gp = ctypes.POINTER(_Geom)
    i, d = ctypes.c_int, ctypes.c_double
    sig = {
        "og_radius": (i, [d, d]),
        "og_taps": (None, [d, i, dp]),
        "og_dims_array": (None, [gp, ip]),
        "og_los": (None, [dp, d, d, dp, dp]),
        "og_los_grid": (None, [dp, i, dp, dp, dp, dp]),
        "og_model_cube": (None, [gp, dp, dp]),
        "og_conv3d_direct": (None, [dp, i, i, i, dp, i, dp, i, dp, i, dp]),
        "og_conv3d_separable": (None, [dp, i, i, i, dp, i, dp, i, dp, i, dp]),
        "og_downsample": (None, [dp, i, i, i, i, dp]),
        "og_moments": (None, [dp, i, i, i, d, d, d, d, dp]),
        "og_eval": (None, [gp, dp, dp, dp]),
        "og_chi2_maps": (d, [dp, i, fp, fp, fp, fp, up, dp]),
        "og_eval_batch": (None, [gp, i, dp, dp, i]),
        "og_chi2_batch": (None, [gp, i, dp, fp, fp, fp, fp, up, dp, dp, i]),
        "og_max_threads": (i, []),
        "og_set_conv_form": (None, [i]),
        "og_get_conv_form": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _u(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def dims(g: Geom):
    """(u, nxf, nyf, nzf, rxy, rz, exf, eyf, ezf) of the fine extended grid."""
    out = np.zeros(9, dtype=np.int32)
    gc = g.c()
    lib().og_dims_array(ctypes.byref(gc), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return tuple(int(v) for v in out)


def radius(sigma, halo=4.0):
    return lib().og_radius(float(sigma), float(halo))


def taps(sigma, R):
    w = np.zeros(2 * R + 1)
    lib().og_taps(float(sigma), int(R), _d(w))
    return w


def los(p, x, y):
    """Line-of-sight velocity and surface brightness at positions (x, y)."""
    p = _c64(p)
    xb, yb = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
    shape = xb.shape
    x, y = _c64(xb).ravel(), _c64(yb).ravel()
    v = np.zeros(x.size)
    b = np.zeros(x.size)
    lib().og_los_grid(_d(p), x.size, _d(x), _d(y), _d(v), _d(b))
    return v.reshape(shape), b.reshape(shape)


def model_cube(g: Geom, p):
    """Fine extended model cube [ezf][eyf][exf]."""
    u, nxf, nyf, nzf, rxy, rz, ex, ey, ez = dims(g)
    out = np.zeros((ez, ey, ex))
    gc = g.c()
    lib().og_model_cube(ctypes.byref(gc), _d(_c64(p)), _d(out))
    return out


def conv3d(ext, wx, wy, wz, separable=False):
    ext = _c64(ext)
    ez, ey, ex = ext.shape
    rx, ry, rz = (len(wx) - 1) // 2, (len(wy) - 1) // 2, (len(wz) - 1) // 2
    out = np.zeros((ez - 2 * rz, ey - 2 * ry, ex - 2 * rx))
    f = lib().og_conv3d_separable if separable else lib().og_conv3d_direct
    f(_d(ext), ex, ey, ez, _d(_c64(wx)), rx, _d(_c64(wy)), ry, _d(_c64(wz)), rz, _d(out))
    return out


def downsample(fine, u):
    fine = _c64(fine)
    nz, ny, nx = fine.shape[0] // u, fine.shape[1] // u, fine.shape[2] // u
    out = np.zeros((nz, ny, nx))
    lib().og_downsample(_d(fine), u, nx, ny, nz, _d(out))
    return out


def moments(cube, dv, vc=0.0, scale=1.0, v_invalid=0.0):
    cube = _c64(cube)
    nz, ny, nx = cube.shape
    maps = np.zeros((3, ny, nx))
    lib().og_moments(_d(cube), nx, ny, nz, float(dv), float(vc), float(scale),
                     float(v_invalid), _d(maps))
    return maps


def evaluate(g: Geom, p, want_cube=False):
    """Model cube (data resolution, optional) and maps [3][ny][nx]."""
    p = _c64(p)
    maps = np.zeros((3, g.ny, g.nx))
    cube = np.zeros((g.nz, g.ny, g.nx)) if want_cube else None
    gc = g.c()
    lib().og_eval(ctypes.byref(gc), _d(p), _d(cube) if want_cube else None, _d(maps))
    return (cube, maps) if want_cube else maps


def evaluate_batch(g: Geom, params, nthreads=0):
    params = _c64(params).reshape(-1, NPAR)
    n = params.shape[0]
    maps = np.zeros((n, 3, g.ny, g.nx))
    gc = g.c()
    lib().og_eval_batch(ctypes.byref(gc), n, _d(params), _d(maps), int(nthreads))
    return maps


@dataclass
class Obs:
    """Observed maps (FP32, [ny][nx]) and uint8 mask; w_v = 1/E_v and
    w_s = sqrt(W)/E_s."""
    v: np.ndarray
    s: np.ndarray
    w_v: np.ndarray
    w_s: np.ndarray
    mask: np.ndarray

    def arrays(self):
        return (_c32(self.v), _c32(self.s), _c32(self.w_v), _c32(self.w_s),
                np.ascontiguousarray(self.mask, dtype=np.uint8))


def chi2_maps(maps, obs: Obs, want_resid=False):
    maps = _c64(maps)
    np_ = maps.shape[-1] * maps.shape[-2]
    v, s, wv, ws, m = obs.arrays()
    resid = np.zeros((2,) + maps.shape[-2:]) if want_resid else None
    c = lib().og_chi2_maps(_d(maps), np_, _f(v), _f(s), _f(wv), _f(ws), _u(m),
                           _d(resid) if want_resid else None)
    return (c, resid) if want_resid else c


def chi2_batch(g: Geom, params, obs: Obs, want_resid=False, nthreads=0):
    params = _c64(params).reshape(-1, NPAR)
    n = params.shape[0]
    v, s, wv, ws, m = obs.arrays()
    chi2 = np.zeros(n)
    resid = np.zeros((n, 2, g.ny, g.nx)) if want_resid else None
    gc = g.c()
    lib().og_chi2_batch(ctypes.byref(gc), n, _d(params), _f(v), _f(s), _f(wv), _f(ws), _u(m),
                        _d(chi2), _d(resid) if want_resid else None, int(nthreads))
    return (chi2, resid) if want_resid else chi2


def max_threads():
    return lib().og_max_threads()


class separable_convolution:
    """Context manager: inside it every evaluation convolves with the three
    1-D passes (``og_conv3d_separable``) instead of the direct 3-D sum.  The
    two forms are the same linear map (pinned term by term on small cubes and
    on whole models); the passes make sweeps over 10^5 models affordable."""

    def __enter__(self):
        self._prev = lib().og_get_conv_form()
        lib().og_set_conv_form(1)
        return self

    def __exit__(self, *exc):
        lib().og_set_conv_form(self._prev)
        return False
