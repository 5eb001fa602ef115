"""Nested sampling (Sec. 2.3.2): the GPU sampler (gbk_nested_sample) compared
with the oracle's on the disc model statistically (both are randomised) and
against the truth.  The oracle's sampler itself is pinned on a Gaussian
likelihood whose evidence is known in closed form (tests/fit_pins.py)."""
import math

import numpy as np
import pytest

import oracle
from oracle import fit
from cases import ogeom
from paper_1510_01815_gb300 import synth
from paper_1510_01815_gb300.synth import Geometry, params as P


GEOM = Geometry(16, 16, 24, 20.0, 0.0, 2.5, 30.0)
TRUTH = P(7.6, 7.4, 50.0, 55.0, 0.0, 160.0, 2.5, 35.0, 1.0, 3.0)


def _box():
    lo, hi = TRUTH.copy(), TRUTH.copy()
    lo[synth.PA], hi[synth.PA] = 20.0, 80.0
    lo[synth.INCL], hi[synth.INCL] = 30.0, 80.0
    lo[synth.VMAX], hi[synth.VMAX] = 80.0, 260.0
    return lo, hi


def _obs():
    m = oracle.evaluate(ogeom(GEOM), TRUTH)
    rng = np.random.default_rng(3)
    shape = (GEOM.ny, GEOM.nx)
    wv, ws = synth.weights(shape, 5.0)
    return oracle.Obs((m[1] + rng.normal(0, 5, shape)).astype(np.float32),
                      (m[2] + rng.normal(0, 7.07, shape)).astype(np.float32), wv, ws, np.ones(shape, np.uint8))


@pytest.mark.gpu
def test_gpu_sampler_agrees_with_oracle_sampler():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    obs = _obs()
    lo, hi = _box()
    ro = fit.nested_sample_model(ogeom(GEOM), obs, lo, hi, n_live=50, batch=12, tol=0.5, seed=11)
    dobs = gbk.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    rg = gbk.gbk_nested_sample(GEOM, dobs, lo, hi, n_live=50, batch=12, tol=0.5, seed=11)
    for k in (synth.PA, synth.INCL, synth.VMAX):
        # posterior means agree within the posterior width and contain the truth
        assert abs(rg["mean"][k] - ro["mean"][k]) < 1.5 * max(ro["std"][k], rg["std"][k]) + 1e-6, k
        assert abs(rg["mean"][k] - TRUTH[k]) < 4 * rg["std"][k] + 0.5, (k, rg["mean"][k], rg["std"][k])
    err = math.sqrt(max(ro["info"], 1e-3) / 50)
    assert abs(rg["log_z"] - ro["log_z"]) < 6 * err, (rg["log_z"], ro["log_z"], err)
    assert rg["n_eval"] > 50 and rg["n_iter"] > 0
