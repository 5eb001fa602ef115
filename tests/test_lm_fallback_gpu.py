"""LM from a learned start with the plain fit as its fallback
(gbk_fit_lm_fallback): seeds that land in the wrong minimum are refitted
from the Sec. 2.1.9 starting point, good seeds are left as gbk_fit_lm
returns them."""
import numpy as np
import pytest
import torch

from cases import noisy_mocks
from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu

G1 = synth.SINGLE_GEOM
FREE = (0, 1, 2, 3, 4, 5, 6, 7)


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def _bounds(truth):
    lo, hi = truth.copy(), truth.copy()
    lo[:, 0], hi[:, 0] = 0.0, G1.nx - 1.0
    lo[:, 1], hi[:, 1] = 0.0, G1.ny - 1.0
    lo[:, 2], hi[:, 2] = -360.0, 720.0
    lo[:, 3], hi[:, 3] = 1.0, 89.0
    lo[:, 4], hi[:, 4] = -200.0, 200.0
    lo[:, 5], hi[:, 5] = 1.0, 600.0
    lo[:, 6], hi[:, 6] = 0.05, 30.0
    lo[:, 7], hi[:, 7] = 1.0, 300.0
    return lo, hi


@pytest.fixture(scope="module")
def case(G):
    n = 32
    truth, cont, obs = noisy_mocks(G1, n, 11)
    dobs = [G.Obs.from_numpy(o.v, o.s, o.w_v, o.w_s, o.mask) for o in obs]
    lo, hi = _bounds(truth)
    rng = np.random.default_rng(12)
    seed = np.array([synth.perturb(rng, truth[i], FREE, 0.05, lo[i], hi[i]) for i in range(n)])
    bad = np.zeros(n, bool)
    bad[1::2] = True
    seed[bad, 2] += 180.0  # the mirrored field: LM stays in the wrong minimum
    heur = np.clip(G.initial_guess(G1, dobs, truth, continuum=cont), lo, hi)
    nres = np.array([2.0 * np.count_nonzero(o.mask) for o in obs])
    return truth, dobs, lo, hi, seed, bad, heur, nres


def _first_and_fallback(G, dobs, seed, heur, lo, hi, opts, refit):
    """gbk_fit_lm from the seeds, and gbk_fit_lm from the fallback starts of
    the galaxies `refit` (in index order, as the library packs them)."""
    q0, c0, it0, st0 = G.fit_lm(G1, dobs, seed, lo, hi, opts)
    sel = np.flatnonzero(refit)
    qb, cb, itb, stb = G.fit_lm(G1, [dobs[i] for i in sel], heur[sel], lo[sel], hi[sel], opts)
    return (q0, c0, it0, st0), sel, (qb, cb, itb, stb)


def test_forced_fallback_keeps_the_lower_chi2(G, case):
    truth, dobs, lo, hi, seed, bad, heur, nres = case
    opts = G.lm_opts(max_iter=200)
    acc = np.where(bad, 0.0, np.inf)  # every flipped seed is refitted
    q, c, it, st, used = G.fit_lm_fallback(G1, dobs, seed, heur, lo, hi, opts, chi2_accept=acc)
    q0, c0, it0, st0 = G.fit_lm(G1, dobs, seed, lo, hi, opts)
    refit = bad | ~np.isin(st0, [1, 2])
    assert np.array_equal(used > 0, refit)
    (q0, c0, it0, st0), sel, (qb, cb, itb, stb) = _first_and_fallback(G, dobs, seed, heur, lo, hi, opts, refit)
    keep = used == 0
    np.testing.assert_allclose(q[keep], q0[keep], rtol=1e-12, atol=1e-12)
    np.testing.assert_array_equal(c[keep], c0[keep])
    take_b = cb < c0[sel]
    assert np.array_equal(used[sel], np.where(take_b, 1, 2))
    np.testing.assert_allclose(c[sel], np.where(take_b, cb, c0[sel]), rtol=1e-9)
    np.testing.assert_allclose(q[sel], np.where(take_b[:, None], qb, q0[sel]), rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(it[sel], np.where(take_b, itb, it0[sel]))
    assert G.gbk_device_status() == 0


def test_wrong_minima_fall_back_under_a_chi2_bound(G, case):
    truth, dobs, lo, hi, seed, bad, heur, nres = case
    opts = G.lm_opts(max_iter=200)
    q0, c0, it0, st0 = G.fit_lm(G1, dobs, seed, lo, hi, opts)
    acc = 1.5 * nres
    q, c, it, st, used = G.fit_lm_fallback(G1, dobs, seed, heur, lo, hi, opts, chi2_accept=acc)
    refit = ~np.isin(st0, [1, 2]) | ~(c0 <= acc)
    assert np.array_equal(used > 0, refit)
    # seeds with PA flipped by 180 degrees end in the mirrored minimum (V_t or
    # i driven down), far above the noise level
    assert refit[bad].sum() >= 4, c0[bad] / nres[bad]
    assert np.all(c <= c0)
    # most refitted galaxies reach the noise level from the Sec. 2.1.9 start
    fixed = (used == 1)
    dpa = np.abs((q[:, 2] - truth[:, 2] + 180.0) % 360.0 - 180.0)
    good = (c <= acc) & (dpa < 3.0)
    assert fixed.sum() >= 4 and good[fixed].mean() >= 0.75, (c[fixed] / nres[fixed], dpa[fixed])


def test_without_a_chi2_bound_only_unconverged_fits_fall_back(G, case):
    truth, dobs, lo, hi, seed, bad, heur, nres = case
    opts = G.lm_opts(max_iter=200)
    q0, c0, it0, st0 = G.fit_lm(G1, dobs, seed, lo, hi, opts)
    q, c, it, st, used = G.fit_lm_fallback(G1, dobs, seed, heur, lo, hi, opts)
    conv = np.isin(st0, [1, 2])
    assert np.array_equal(used > 0, ~conv)
    np.testing.assert_array_equal(c[conv], c0[conv])
