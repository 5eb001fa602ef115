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


# Trajectory parity.  Both samplers implement the same algorithm with the same
# SplitMix64 stream, so with the same seed they draw the same initial live
# points and the same proposals, and make the same replacements, for as long
# as every replacement decision comes out the same way.  A decision compares
# a proposal's chi2 with the worst live point's.  The GPU's chi2 of a model
# differs from the oracle's by what its FP32 maps imply (at most 1e-4
# relative here, checked for every point); the two samplers decide alike
# whenever the oracle's gap exceeds the two points' GPU-oracle differences,
# so a decision within twice that is a near-tie.  The comparison stops at the
# first near-tie (the trajectories may part there for good); before it
# everything must agree.
CHI2_REL = 1e-4


@pytest.mark.gpu
def test_gpu_sampler_trajectory_matches_oracle():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    obs = _obs()
    lo, hi = _box()
    n_live, batch, iters, seed = 50, 12, 60, 23
    tr_o = {}
    fit.nested_sample_model(ogeom(GEOM), obs, lo, hi, n_live=n_live, batch=batch, tol=1e-9, seed=seed,
                            max_iter=iters, trace=tr_o)
    dobs = gbk.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    rg = gbk.gbk_nested_sample_traced(GEOM, dobs, lo, hi, n_live=n_live, batch=batch, tol=1e-9, seed=seed,
                                      max_iter=iters, trace_iters=iters)
    tg = rg["trace"]
    # initial live points: the same draws (FP64, up to contraction of a*b+c)
    np.testing.assert_allclose(tg["live0"], tr_o["live0"], rtol=1e-14, atol=0)
    np.testing.assert_allclose(tg["live0_chi2"], -2.0 * tr_o["live0_logl"], rtol=CHI2_REL)
    # the live sets' chi2 (oracle, GPU), replayed with the common decisions
    c_o = -2.0 * tr_o["live0_logl"]
    c_g = np.array(tg["live0_chi2"], dtype=np.float64)
    assert len(tg["n_props"]) == len(tr_o["props"]) == iters
    compared = replaced = 0
    for t in range(iters):
        props_o, pc_o, repl_o = tr_o["props"][t], -2.0 * tr_o["logl"][t], tr_o["replaced"][t]
        k = int(tg["n_props"][t])
        assert k == len(props_o), (t, k, len(props_o))
        np.testing.assert_allclose(tg["props"][t][:k], props_o, rtol=1e-9, atol=1e-9)
        pc_g = tg["chi2"][t][:k]
        np.testing.assert_allclose(pc_g, pc_o, rtol=CHI2_REL)
        tie = False
        for j in range(k):
            order = np.argsort(-c_o, kind="stable")
            w, w2 = int(order[0]), int(order[1])  # worst live point = largest chi2, and the runner-up
            err = np.abs(c_g - c_o)
            if c_o[w] - c_o[w2] <= 2.0 * (err[w] + err[w2]) + 1e-12 * c_o[w]:
                tie = True  # which point is the worst is itself undecided
                break
            gap = abs(pc_o[j] - c_o[w])
            if gap <= 2.0 * (abs(pc_g[j] - pc_o[j]) + err[w]) + 1e-12 * c_o[w]:
                tie = True
                break
            assert tg["replaced"][t][j] == repl_o[j], (t, j, tg["replaced"][t][j], repl_o[j])
            if repl_o[j] >= 0:
                c_o[w], c_g[w] = pc_o[j], pc_g[j]
                replaced += 1
        if tie:
            print("near-tie at iteration %d; %d iterations compared" % (t, compared))
            break
        compared += 1
    # a trajectory long enough to have shrunk the prior volume many times
    assert compared >= 30, compared
    assert replaced >= 100, replaced


# The Fabry-Perot workload at reduced size (48 x 48 x 48 at 10 km/s, PSF FWHM
# 3 px, LSF 30 km/s), noiseless maps, 400 live points and 100 proposals per
# launch as in the full workload, the five parameters of its prior free over
# its ranges: the posterior mean of each lies within two posterior standard
# deviations of the truth.
FP48 = Geometry(48, 48, 48, 10.0, 0.0, 3.0, 30.0)


@pytest.mark.gpu
def test_gpu_sampler_fabry_perot_48_noiseless_recovers_truth():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    truth = P(23.7, 23.2, 130.0, 52.0, 0.0, 180.0, 3.0, 30.0, 1.0, 5.0)
    m = oracle.evaluate(ogeom(FP48), truth)
    shape = (FP48.ny, FP48.nx)
    wv, ws = synth.weights(shape, 5.0)
    mask = synth.sn_mask(m[0], 3.0, 0.01).astype(np.uint8)
    dobs = gbk.Obs.from_numpy(m[1].astype(np.float32), m[2].astype(np.float32), wv, ws, mask)
    lo, hi = truth.copy(), truth.copy()
    for k, (a, b) in synth.FP_RANGES.items():
        lo[k], hi[k] = a, b
    r = gbk.gbk_nested_sample(FP48, dobs, lo, hi, n_live=400, batch=100, tol=0.5, seed=5)
    for k in synth.FP_RANGES:
        assert abs(r["mean"][k] - truth[k]) <= 2.0 * r["std"][k] + 1e-9, (k, r["mean"][k], r["std"][k], truth[k])
        assert r["std"][k] < 0.05 * (hi[k] - lo[k]), (k, r["std"][k])
    assert r["n_eval"] > 400 and np.isfinite(r["log_z"])
