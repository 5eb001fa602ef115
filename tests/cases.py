"""Parity cases shared by the GPU tests: seeded inputs (from synth), expected
values from the FP64 oracle, and the tolerances the comparisons use.

Tolerances (maps 1e-4 relative, with scales for values near zero):
  |dm1| <= 1e-4 * max(|m1_ref|, Vmax)
  |dm2| <= 1e-4 * max(m2_ref, sigma0)
  |dm0| <= 1e-4 * max(m0_ref)
A spectrum's validity (m0 > 1e-20 I0) must agree except where the oracle's
m0 / I0 lies within a factor 2 of the threshold (an FP32 vs FP64 decision).
The end-to-end chi2 may differ by what the measured map deviations imply,
sum 2 |r| |w d| + (w d)^2, plus 1e-6 relative for the FP32 residuals.
"""
import numpy as np

import oracle
from paper_1510_01815_gb300 import synth

THRESH = 1e-20


def ogeom(g):
    return oracle.Geom(**g.asdict())


def make_obs(g, p_true, seed, noise_v=5.0, dead=0.02, sn_eta=None):
    """Observed maps from the oracle at p_true plus seeded noise; weights
    1/E_v and 1/(sqrt(2) E_v); dead-fibre mask (and S/N mask if sn_eta)."""
    rng = np.random.default_rng(seed)
    m = oracle.evaluate(ogeom(g), p_true)
    shape = (g.ny, g.nx)
    v = m[1] + synth.gaussian_noise(rng, shape, noise_v)
    s = m[2] + synth.gaussian_noise(rng, shape, noise_v * np.sqrt(2.0))
    wv, ws = synth.weights(shape, noise_v)
    mask = synth.dead_fibre_mask(rng, shape, dead)
    if sn_eta is not None:
        mask = mask * synth.sn_mask(m[0], 3.0, sn_eta)
    return oracle.Obs(v.astype(np.float32), s.astype(np.float32), wv, ws, mask.astype(np.uint8))


def model_params(g, p_true, n, seed, frac=0.2):
    rng = np.random.default_rng(seed)
    ps = [p_true] + [synth.perturb(rng, p_true, frac=frac) for _ in range(n - 1)]
    return np.array(ps)


def check_maps(gpu, ref, params, label=""):
    """gpu, ref: [n][3][ny][nx]; params [n][10]."""
    gpu = np.asarray(gpu, dtype=np.float64)
    n = ref.shape[0]
    worst = 0.0
    for i in range(n):
        p = params[i]
        i0, vmax, s0 = p[synth.I0], abs(p[synth.VMAX]), p[synth.SIG0]
        r0, r1, r2 = ref[i]
        g0, g1, g2 = gpu[i]
        vr = r0 > 0
        vg = g0 > 0
        border = (r0 > 0.5 * THRESH * i0) & (r0 < 2.0 * THRESH * i0)
        bad = (vr != vg) & ~border
        assert not bad.any(), "%s model %d: validity differs at %s" % (label, i, np.argwhere(bad)[:5])
        both = vr & vg
        e0 = np.abs(g0 - r0)[both] / max(r0.max(), 1e-300)
        e1 = np.abs(g1 - r1)[both] / np.maximum(np.abs(r1[both]), vmax)
        e2 = np.abs(g2 - r2)[both] / np.maximum(r2[both], s0)
        for name, e in (("m0", e0), ("m1", e1), ("m2", e2)):
            if e.size:
                worst = max(worst, float(e.max()))
                assert e.max() <= 1e-4, "%s model %d %s: max rel err %.3g" % (label, i, name, e.max())
        inv = ~vr & ~border & ~vg
        if inv.any():
            assert np.all(g0[inv] == 0) and np.all(g2[inv] == 0)
            np.testing.assert_allclose(g1[inv], p[synth.VSYS], rtol=0, atol=1e-4 * max(vmax, 1.0))
    return worst


def chi2_bound(ref_maps, gpu_maps, obs, ref_chi2):
    """Bound on |chi2_gpu - chi2_ref| implied by the map deviations."""
    ref_maps = np.asarray(ref_maps, dtype=np.float64)
    gpu_maps = np.asarray(gpu_maps, dtype=np.float64)
    use = (obs.mask != 0) & (ref_maps[0] > 0)
    b = 0.0
    for k, ob, w in ((1, obs.v, obs.w_v), (2, obs.s, obs.w_s)):
        r = w * (ref_maps[k] - ob)
        d = w * (gpu_maps[k] - ref_maps[k])
        b += float(np.sum((2 * np.abs(r) * np.abs(d) + d * d)[use]))
    return b + 1e-6 * abs(ref_chi2) + 1e-9


def noisy_mocks(g, n, seed, noise=5.0):
    """n single-galaxy mocks of geometry g: parameters drawn around the
    image centre, oracle maps plus seeded noise (noise on v, sqrt(2) noise
    on sigma) and a dead-fibre mask.  Returns (truth [n][10], continuum
    maps [n][ny][nx] FP32, [oracle.Obs])."""
    import math
    rng = np.random.default_rng(seed)
    truth, cont, obs = [], [], []
    for _ in range(n):
        p = synth.params(rng.uniform(0.4, 0.6) * (g.nx - 1), rng.uniform(0.4, 0.6) * (g.ny - 1),
                         rng.uniform(0.0, 360.0), rng.uniform(25.0, 70.0), rng.uniform(-20.0, 20.0),
                         rng.uniform(100.0, 250.0), rng.uniform(1.5, 4.0), rng.uniform(20.0, 60.0), 1.0,
                         rng.uniform(3.0, 6.0))
        m = oracle.evaluate(ogeom(g), p)
        shape = (g.ny, g.nx)
        v = (m[1] + rng.normal(0.0, noise, shape)).astype(np.float32)
        s_ = (m[2] + rng.normal(0.0, noise * math.sqrt(2.0), shape)).astype(np.float32)
        wv, ws = synth.weights(shape, max(noise, 1.0))
        mask = synth.dead_fibre_mask(rng, shape).astype(np.uint8)
        truth.append(p)
        cont.append(m[0].astype(np.float32))
        obs.append(oracle.Obs(v, s_, wv, ws, mask))
    return np.array(truth), np.array(cont), obs
