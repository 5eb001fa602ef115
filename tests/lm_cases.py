"""Shared set-up of the Levenberg-Marquardt tests: the single-galaxy workload
(32 x 32 x 64, Sec. 3.1 mock resolution), observed maps from the oracle at
the true parameters, bounds and perturbed starts."""
import numpy as np

import oracle
from paper_1510_01815_gb300 import synth
from cases import ogeom

FREE = synth.FREE_DEFAULT


def bounds(p):
    lo = np.array(p, dtype=np.float64)
    hi = np.array(p, dtype=np.float64)
    lo[synth.X0], hi[synth.X0] = 0.0, 31.0
    lo[synth.Y0], hi[synth.Y0] = 0.0, 31.0
    lo[synth.PA], hi[synth.PA] = -360.0, 720.0
    lo[synth.INCL], hi[synth.INCL] = 1.0, 89.0          # Sec. 3.1 fitting bounds
    lo[synth.VSYS], hi[synth.VSYS] = -200.0, 200.0
    lo[synth.VMAX], hi[synth.VMAX] = 1.0, 600.0
    lo[synth.RT], hi[synth.RT] = 0.05, 30.0
    lo[synth.SIG0], hi[synth.SIG0] = 1.0, 300.0
    return lo, hi


def galaxy(noise_v=0.0, seed=1, truth=None):
    g = synth.SINGLE_GEOM
    p = synth.SINGLE_TRUTH.copy() if truth is None else np.asarray(truth, dtype=np.float64)
    m = oracle.evaluate(ogeom(g), p)
    rng = np.random.default_rng(seed)
    shape = (g.ny, g.nx)
    e_v = 5.0
    v = m[1] + (rng.normal(0, noise_v, shape) if noise_v > 0 else 0.0)
    s = m[2] + (rng.normal(0, noise_v * np.sqrt(2), shape) if noise_v > 0 else 0.0)
    wv, ws = synth.weights(shape, e_v)
    return g, p, oracle.Obs(v.astype(np.float32), s.astype(np.float32), wv, ws, np.ones(shape, np.uint8))


def starts(p, n, seed=2, frac=0.2):
    rng = np.random.default_rng(seed)
    lo, hi = bounds(p)
    return np.array([synth.perturb(rng, p, FREE, frac, lo, hi) for _ in range(n)])
