"""Pins of the optimisers of Sec. 2.3 over the FP64 oracle (oracle/fit.py) as
functions of the module under test, so that the same pins check the oracle
and the mistakes planted in copies of it.  Each raises AssertionError when
violated.  They test it against what fixes the answer independently:

  LM   -- noiseless data has its chi2 minimum at the truth (Sec. 4.1's
          thresholds from perturbed starts); with only V_sys free the
          residual is linear in it, so the first (lightly damped) step is
          exact and the gain ratio is 1 (lambda / 10 per step: a closed
          form for the offset); a fully masked galaxy rejects every step
          (lambda x 2, 4, 8, ...: the stop at a known iteration); an optimum
          outside the box ends on the box's face;
  NG   -- a truth placed on a node is the unique zero-chi2 node, at its
          row-major index; every node's chi2 is the direct evaluation at the
          node's value; invalid (NaN) nodes lose to finite ones; the next
          level's nodes are the documented box around the best node;
  NS   -- SplitMix64's published first outputs; the closed-form evidence of
          a Gaussian likelihood in a box; the recorded trajectory replays
          as the run; L = 0 outside the parameter domain."""
import math

import numpy as np

import oracle
from cases import ogeom
from lm_cases import FREE, bounds, galaxy, starts
from paper_1510_01815_gb300 import synth
from paper_1510_01815_gb300.synth import Geometry, params as P

# the nested-grid case: the truth sits on node (PA 2, i 2, Vmax 2, rt 1, sig 1)
GRID_GEOM = Geometry(24, 24, 32, 20.0, 0.0, 2.5, 30.0)
GRID_TRUTH = P(11.5, 11.5, 60.0, 50.0, 0.0, 180.0, 3.0, 40.0, 1.0, 4.0)
GRID_NODES = [1, 1, 5, 4, 1, 5, 3, 3, 1, 1]
GRID_LO = GRID_TRUTH.copy()
GRID_HI = GRID_TRUTH.copy()
GRID_LO[2], GRID_HI[2] = 40.0, 80.0   # step 10
GRID_LO[3], GRID_HI[3] = 30.0, 60.0   # step 10
GRID_LO[5], GRID_HI[5] = 140.0, 220.0  # step 20
GRID_LO[6], GRID_HI[6] = 2.0, 4.0     # step 1
GRID_LO[7], GRID_HI[7] = 30.0, 50.0   # step 10
GRID_TRUTH_INDEX = (((2 * 4 + 2) * 5 + 2) * 3 + 1) * 3 + 1


def grid_noiseless_obs():
    m = oracle.evaluate(ogeom(GRID_GEOM), GRID_TRUTH)
    wv, ws = synth.weights((GRID_GEOM.ny, GRID_GEOM.nx), 5.0)
    return oracle.Obs(m[1].astype(np.float32), m[2].astype(np.float32), wv, ws,
                      np.ones((GRID_GEOM.ny, GRID_GEOM.nx), np.uint8))


def pin_splitmix64_reference_values(fit):
    r = fit.SplitMix64(0)
    assert [r.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def pin_sampler_gaussian_evidence(fit):
    """exp(-|x - m|^2 / 2 s^2) in a box of volume V >> s^d: Z = (2 pi s^2)^(d/2)
    / V; log Z within 3 sqrt(H / N) plus the shrinkage's discretisation, the
    posterior mean m and standard deviation s within 15 percent."""
    d, s = 3, 0.3
    m = np.array([0.4, -0.2, 0.1])
    lo = np.zeros(10)
    hi = np.zeros(10)
    lo[:d], hi[:d] = -2.0, 2.0
    V = 4.0 ** d

    def loglike(p):
        x = p[:, :d] - m
        return -0.5 * np.sum(x * x, axis=1) / (s * s)

    N = 100
    # the run stops by its evidence tolerance after about 60 iterations; the
    # cap only bounds a broken sampler's run
    r = fit.nested_sample(loglike, lo, hi, n_live=N, batch=25, tol=0.01, seed=7, max_iter=2000)
    assert r["n_iter"] < 2000, r["n_iter"]
    true_lz = 0.5 * d * math.log(2 * math.pi * s * s) - math.log(V)
    err = math.sqrt(max(r["info"], 1e-3) / N)
    assert abs(r["log_z"] - true_lz) < 3 * err + 0.05, (r["log_z"], true_lz, err)
    np.testing.assert_allclose(r["mean"][:d], m, atol=0.15 * s + 0.02)
    np.testing.assert_allclose(r["std"][:d], s, rtol=0.15)


def pin_lm_solves_a_linear_problem_in_one_step(fit):
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    p0 = p.copy()
    p0[synth.VSYS] = 25.0
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, [synth.VSYS], max_iter=1, fd_step=0.1)
    assert abs(q[synth.VSYS]) < 25.0 * 2e-3, q[synth.VSYS]


def pin_lm_central_differences_solve_the_linear_problem(fit):
    """The same linear problem with central differences: (r(p + h) - r(p -
    h)) / 2h of a linear residual is its exact slope, so the first step lands
    within the damping's 0.1 percent as well."""
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    p0 = p.copy()
    p0[synth.VSYS] = 25.0
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, [synth.VSYS], max_iter=1, fd_step=0.1, central=True)
    assert abs(q[synth.VSYS]) < 25.0 * 2e-3, q[synth.VSYS]


def pin_lm_gain_ratio_on_a_linear_problem(fit):
    """With only V_sys free the residual is linear in it, so the linearised
    model predicts each step's chi2 decrease exactly: the gain ratio is 1 and
    every step divides lambda by ten.  A damped step from offset x leaves
    x lambda / (1 + lambda), so from lambda0 = 1e4 six steps leave
    25 prod_j lambda_j / (1 + lambda_j) km/s, lambda_j = 1e4 / 10^j (1.02 km/s;
    a damping that stayed at 1e4 would leave 24.99)."""
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    p0 = p.copy()
    p0[synth.VSYS] = p[synth.VSYS] + 25.0
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, [synth.VSYS], max_iter=6, fd_step=0.1, lambda0=1e4)
    lam = 1e4 / 10.0 ** np.arange(6)
    want = 25.0 * np.prod(lam / (1.0 + lam))
    assert it == 6, (it, st)
    assert abs((q[synth.VSYS] - p[synth.VSYS]) - want) < 1e-4 * want + 1e-5, (q[synth.VSYS] - p[synth.VSYS], want)


def pin_lm_masked_galaxy_rejects_every_step(fit):
    """Every spaxel masked: chi2 is 0 whatever the parameters, J = 0, the
    damped step is zero and every trial is rejected, so lambda grows by nu =
    2, 4, 8, ... from 1e-3: 1e-3 x 2^(k (k + 1) / 2) first exceeds 1e12 at
    the 10th iteration, where the fit stops (status LAMBDA) at its start."""
    g, p, obs = galaxy(noise_v=0.0)
    obs = oracle.Obs(obs.v, obs.s, obs.w_v, obs.w_s, np.zeros_like(obs.mask))
    lo, hi = bounds(p)
    p0 = starts(p, 1, seed=5)[0]
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, FREE, max_iter=50, lambda0=1e-3)
    assert (it, st) == (10, 4), (it, st)
    assert np.array_equal(q, p0)


def pin_lm_optimum_outside_the_box_ends_on_its_face(fit):
    """Noiseless data with V_max = 200 fitted with V_max free and capped at
    180: chi2 falls monotonically towards the cap, so the fit ends exactly on
    it (the trial points are clipped to the box)."""
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    hi[synth.VMAX] = 180.0
    p0 = p.copy()
    p0[synth.VMAX] = 150.0
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, [synth.VMAX], max_iter=60)
    assert q[synth.VMAX] == 180.0, q[synth.VMAX]


def pin_lm_recovers_noiseless_parameters(fit):
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    for p0 in starts(p, 2, seed=3):
        q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, FREE, max_iter=100)
        assert st in (1, 2), (st, it)  # FTOL, XTOL
        assert abs(q[synth.VMAX] - p[synth.VMAX]) < 2.0, q
        assert abs(q[synth.PA] - p[synth.PA]) < 1.0, q
        assert c < 1e-6, c


def pin_grid_row_major_order(fit):
    """A 1-D grid over PA: chi2 per node equals the direct evaluation at the
    node's value, in order."""
    obs = grid_noiseless_obs()
    nodes = [1] * 10
    nodes[2] = 7
    lo, hi = GRID_TRUTH.copy(), GRID_TRUTH.copy()
    lo[2], hi[2] = 0.0, 120.0
    bp, bi, bc, allc = fit.grid_search(ogeom(GRID_GEOM), obs, lo, hi, nodes, GRID_TRUTH, levels=1)
    vals = np.array([GRID_TRUTH] * 7)
    vals[:, 2] = np.arange(7) * 20.0
    np.testing.assert_allclose(allc[0], oracle.chi2_batch(ogeom(GRID_GEOM), vals, obs), rtol=1e-12)
    assert bi[0] == 3


def pin_grid_invalid_nodes_lose(fit):
    """A 1-D grid over i from 70 to 100 degrees: the nodes at and above 90
    are outside the parameter domain (NaN chi2) and must lose to every
    finite node."""
    obs = grid_noiseless_obs()
    nodes = [1] * 10
    nodes[3] = 7
    lo, hi = GRID_TRUTH.copy(), GRID_TRUTH.copy()
    lo[3], hi[3] = 70.0, 100.0
    bp, bi, bc, allc = fit.grid_search(ogeom(GRID_GEOM), obs, lo, hi, nodes, GRID_TRUTH, levels=1)
    assert np.all(np.isnan(allc[0][4:])) and np.all(np.isfinite(allc[0][:4]))
    assert bi[0] == int(np.argmin(allc[0][:4])) and math.isfinite(bc[0])


def pin_grid_finds_truth_on_a_node(fit):
    """The truth on a node is the unique zero-chi2 node at its row-major
    index; level 1 spans the best node +- one level-0 step (clipped to the
    box) with the same node counts: its first and last nodes' chi2 equal the
    direct evaluation there."""
    obs = grid_noiseless_obs()
    bp, bi, bc, allc = fit.grid_search(ogeom(GRID_GEOM), obs, GRID_LO, GRID_HI, GRID_NODES, GRID_TRUTH, levels=2)
    assert bi[0] == GRID_TRUTH_INDEX, bi
    assert bc[0] < 1e-8
    assert np.sum(allc[0] < 1e-8) == 1
    nodes = np.array(GRID_NODES)
    steps0 = (GRID_HI - GRID_LO) / np.maximum(nodes - 1, 1)
    lo1 = np.maximum(GRID_LO, GRID_TRUTH - steps0)
    hi1 = np.minimum(GRID_HI, GRID_TRUTH + steps0)
    first, last = GRID_TRUTH.copy(), GRID_TRUTH.copy()
    for k in range(10):
        if nodes[k] > 1:
            first[k], last[k] = lo1[k], hi1[k]
    ref = oracle.chi2_batch(ogeom(GRID_GEOM), np.array([first, last]), obs)
    np.testing.assert_allclose([allc[1][0], allc[1][-1]], ref, rtol=1e-12)
    assert np.all(np.abs(bp - GRID_TRUTH) <= steps0 + 1e-12), bp - GRID_TRUTH


# fastest first: a mutant test stops at the first pin that fails
def pin_sampler_trace_replays(fit):
    """The recorded trajectory is the run: replaying the replacements from
    the initial live points, each proposal either beat the worst live point
    of that moment and took its place, or did not beat it and was dropped;
    every proposal lies inside the prior box."""
    d = 3
    lo, hi = np.zeros(10), np.zeros(10)
    lo[:d], hi[:d] = -2.0, 2.0

    def loglike(p):
        x = p[:, :d] - 0.3
        return -0.5 * np.sum(x * x, axis=1) / 0.09

    tr = {}
    r = fit.nested_sample(loglike, lo, hi, n_live=40, batch=10, tol=1e-6, seed=3, max_iter=30, trace=tr)
    assert r["n_iter"] == 30 and len(tr["props"]) == 30
    logl = tr["live0_logl"].copy()
    np.testing.assert_array_equal(logl, loglike(tr["live0"]))
    n_repl = 0
    for props, lp, repl in zip(tr["props"], tr["logl"], tr["replaced"]):
        assert np.all(props >= lo) and np.all(props <= hi)
        np.testing.assert_array_equal(lp, loglike(props))
        for j in range(len(props)):
            w = int(np.argmin(logl))
            if lp[j] > logl[w]:
                assert repl[j] == w, (j, repl[j], w)
                logl[w] = lp[j]
                n_repl += 1
            else:
                assert repl[j] == -1, (j, repl[j])
    assert n_repl > 50


def pin_sampler_outside_the_domain_has_zero_likelihood(fit):
    """A prior box that reaches past the parameter domain (i up to 100 deg;
    the disc model is undefined at i >= 90) on noiseless data: points outside
    have L = 0, so they are the first replaced and never come back; the
    evidence and the posterior stay finite, the posterior inside the domain."""
    g = Geometry(10, 10, 16, 20.0, 0.0, 2.0, 30.0)
    p = P(4.6, 4.4, 40.0, 60.0, 0.0, 150.0, 2.0, 40.0, 1.0, 3.0)
    m = oracle.evaluate(ogeom(g), p)
    wv, ws = synth.weights((g.ny, g.nx), 5.0)
    obs = oracle.Obs(m[1].astype(np.float32), m[2].astype(np.float32), wv, ws, np.ones((g.ny, g.nx), np.uint8))
    lo, hi = p.copy(), p.copy()
    lo[synth.INCL], hi[synth.INCL] = 30.0, 100.0
    lo[synth.VMAX], hi[synth.VMAX] = 80.0, 250.0
    r = fit.nested_sample_model(ogeom(g), obs, lo, hi, n_live=30, batch=8, tol=0.5, seed=4, max_iter=400)
    assert np.isfinite(r["log_z"]) and np.all(np.isfinite(r["mean"]))
    assert r["mean"][synth.INCL] < 90.0 and abs(r["mean"][synth.INCL] - 60.0) < 5.0, r["mean"][synth.INCL]


ALL_FIT_PINS = [pin_splitmix64_reference_values, pin_sampler_gaussian_evidence,
                pin_lm_solves_a_linear_problem_in_one_step, pin_lm_central_differences_solve_the_linear_problem,
                pin_lm_masked_galaxy_rejects_every_step, pin_lm_gain_ratio_on_a_linear_problem,
                pin_grid_row_major_order, pin_grid_invalid_nodes_lose,
                pin_lm_optimum_outside_the_box_ends_on_its_face, pin_lm_recovers_noiseless_parameters,
                pin_grid_finds_truth_on_a_node, pin_sampler_trace_replays,
                pin_sampler_outside_the_domain_has_zero_likelihood]
