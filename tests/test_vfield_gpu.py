"""The velocity-field strategy (Sec. 2.2.1) on the GPU, with the arctan
(Eq. 6) and Epinat (Eq. 7) rotation curves, against the FP64 oracle: maps,
chi-squared, invalid parameters, fits that recover the truth, nested grids,
and the entry points that must refuse a velocity field."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fit
from cases import check_maps, chi2_bound, ogeom
from paper_1510_01815_gb300 import synth
from paper_1510_01815_gb300.synth import Geometry

pytestmark = pytest.mark.gpu

VF_ARCTAN, VF_EPINAT = 1, 2


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def vgeom(nx, ny, model):
    return Geometry(nx, ny, 1, 10.0, model=model)


def vparams(n, seed, nx, ny, model):
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 10))
    p[:, 0] = rng.uniform(0.3, 0.7, n) * (nx - 1)
    p[:, 1] = rng.uniform(0.3, 0.7, n) * (ny - 1)
    p[:, 2] = rng.uniform(0, 360, n)
    p[:, 3] = rng.uniform(10, 80, n)
    p[:, 4] = rng.uniform(-50, 50, n)
    p[:, 5] = rng.uniform(50, 300, n)
    p[:, 6] = rng.uniform(1, 10, n)
    p[:, 7] = rng.uniform(10, 80, n)
    if model == VF_EPINAT:
        p[:, 8] = rng.uniform(0.3, 3.0, n)   # a
        p[:, 9] = rng.uniform(0.2, 2.0, n)   # g (g < 1 exercises the centre rule)
    else:
        p[:, 8], p[:, 9] = 1.0, 3.0
    # one model centred exactly on a pixel
    p[0, 0], p[0, 1] = float(nx // 2), float(ny // 2)
    return p


@pytest.mark.parametrize("model", [VF_ARCTAN, VF_EPINAT])
@pytest.mark.parametrize("nx,ny", [(33, 29), (128, 96), (7, 1)])
def test_vfield_maps_vs_oracle(G, model, nx, ny):
    g = vgeom(nx, ny, model)
    p = vparams(12, 21 + nx + model, nx, ny, model)
    got = G.eval_maps(g, torch.from_numpy(p)).cpu().numpy()
    ref = np.array([oracle.evaluate(ogeom(g), q) for q in p])
    check_maps(got, ref, p, label="vfield model %d" % model)
    # the centre pixel of model 0 is exactly Vsys
    assert abs(got[0, 1, ny // 2, nx // 2] - p[0, 4]) <= 1e-4 * max(abs(p[0, 4]), 1.0)


@pytest.mark.parametrize("model", [VF_ARCTAN, VF_EPINAT])
def test_vfield_chi2_vs_oracle(G, model):
    nx, ny = 64, 48
    g = vgeom(nx, ny, model)
    p = vparams(20, 31 + model, nx, ny, model)
    truth = p[1]
    m = oracle.evaluate(ogeom(g), truth)
    rng = np.random.default_rng(5)
    wv, ws = synth.weights((ny, nx), 5.0)
    obs = oracle.Obs((m[1] + rng.normal(0, 5, (ny, nx))).astype(np.float32),
                     (m[2] + rng.normal(0, 7, (ny, nx))).astype(np.float32), wv, ws,
                     synth.dead_fibre_mask(rng, (ny, nx)).astype(np.uint8))
    d = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    c, r = G.chi2(g, torch.from_numpy(p), d, want_resid=True)
    got_maps = G.eval_maps(g, torch.from_numpy(p)).cpu().numpy()
    for i in range(len(p)):
        ref_maps = oracle.evaluate(ogeom(g), p[i])
        ref_c = oracle.chi2_maps(ref_maps, obs)
        b = chi2_bound(ref_maps, got_maps[i], obs, ref_c)
        assert abs(float(c[i]) - ref_c) <= b, (i, float(c[i]), ref_c, b)


def test_vfield_invalid_parameters(G):
    g = vgeom(16, 16, VF_EPINAT)
    p = vparams(3, 3, 16, 16, VF_EPINAT)
    p[1, 3] = 90.0          # edge-on: outside 0 <= i < 90
    p[2, 8] = np.nan        # Epinat slope not finite
    maps = G.eval_maps(g, torch.from_numpy(p)).cpu().numpy()
    assert np.isfinite(maps[0]).all()
    assert np.isnan(maps[1]).all() and np.isnan(maps[2]).all()


def test_vfield_refusals(G):
    g = vgeom(16, 16, VF_ARCTAN)
    p = torch.from_numpy(vparams(2, 4, 16, 16, VF_ARCTAN))
    with pytest.raises(G.GbkError):
        G.eval_cubes(g, p)
    o = np.zeros((16, 16), np.float32)
    d = G.Obs.from_numpy(o, o, o + 1, o + 1, np.ones((16, 16), np.uint8))
    with pytest.raises(G.GbkError):
        G.chi2(g, p, d, flags=G.PATH_STAGED)
    with pytest.raises(G.GbkError):
        G.gbk_survey_workspace_bytes([g])


def _vf_obs(G, g, truth, seed, noise=3.0):
    """Oracle field of `truth` plus noise, with a masked block."""
    m = oracle.evaluate(ogeom(g), truth)
    rng = np.random.default_rng(seed)
    wv, ws = synth.weights((g.ny, g.nx), 5.0)
    mask = np.ones((g.ny, g.nx), np.uint8)
    mask[2:5, 3:9] = 0
    v = (m[1] + rng.normal(0, noise, m[1].shape)).astype(np.float32)
    sg = (m[2] + rng.normal(0, noise, m[2].shape)).astype(np.float32)
    return oracle.Obs(v, sg, wv, ws, mask)


def _oracle_vf_jacobian(g, p, obs, steps):
    og = ogeom(g)
    cols = []
    for k in range(10):
        a, b = p.copy(), p.copy()
        a[k] += steps[k]
        b[k] -= steps[k]
        _, r = oracle.chi2_batch(og, np.array([a, b]), obs, want_resid=True)
        cols.append((r[0] - r[1]) / (2 * steps[k]))
    return np.array(cols)  # [10][2][ny][nx]


@pytest.mark.parametrize("model", [VF_ARCTAN, VF_EPINAT])
def test_vfield_jacobian_matches_central_differences(G, model):
    """Analytic Jacobian of the velocity-field residuals (every parameter,
    both curves) against FP64 central differences of the oracle; its J^T J,
    J^T r and chi2 against the J it writes."""
    nx, ny = 40, 34
    g = vgeom(nx, ny, model)
    ps = vparams(3, 21, nx, ny, model)
    ps[0, 0] += 0.37  # keep the centre off the pixel grid for central differences
    obs = _vf_obs(G, g, ps[1], 5)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    jac, jtj, jtv, c2 = G.jacobian(g, torch.from_numpy(ps), dobs, free=tuple(range(10)))
    jac = jac.cpu().numpy()
    steps = np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-4, 1e-3, 1e-5, 1e-5])
    for i in range(ps.shape[0]):
        ref = _oracle_vf_jacobian(g, ps[i], obs, steps)
        used = [k for k in range(10) if model == VF_EPINAT or k not in (8, 9)]
        for k in used:
            scale = np.abs(ref[k]).max() + 1e-6
            err = np.abs(jac[i, k] - ref[k]).max()
            assert err <= 2e-3 * scale + 1e-4, (i, k, err, scale)
        if model == VF_ARCTAN:
            assert np.all(jac[i, 8:] == 0.0)
        # reductions of the rows the kernel wrote
        J = jac[i].reshape(10, -1).astype(np.float64)
        _, r = oracle.chi2_batch(ogeom(g), ps[i:i + 1], obs, want_resid=True)
        r = r[0].reshape(-1)
        np.testing.assert_allclose(jtj[i].cpu().numpy(), J @ J.T, rtol=2e-4, atol=1e-3 * np.abs(J @ J.T).max())
        np.testing.assert_allclose(jtv[i].cpu().numpy(), J @ r, rtol=2e-3, atol=2e-3 * np.abs(J @ r).max())
        assert abs(float(c2[i]) - float(r @ r)) <= 1e-4 * float(r @ r)
    assert G.gbk_device_status() == 0


def _fit_case(G, model, seed, frac, jacobian=None):
    nx, ny = 48, 48
    g = vgeom(nx, ny, model)
    rng = np.random.default_rng(seed)
    truth = np.array([23.4, 24.1, 40.0, 55.0, 10.0, 200.0, 4.0, 30.0, 1.0, 1.0])
    if model == VF_EPINAT:
        truth[8], truth[9] = 1.6, 0.9
    m = oracle.evaluate(ogeom(g), truth)
    wv, ws = synth.weights((ny, nx), 5.0)
    d = G.Obs.from_numpy(m[1].astype(np.float32), m[2].astype(np.float32), wv, ws, np.ones((ny, nx), np.uint8))
    free = (0, 1, 2, 3, 4, 5, 6) + ((8, 9) if model == VF_EPINAT else (7,))
    lo, hi = truth.copy(), truth.copy()
    bounds = {0: (0, nx - 1), 1: (0, ny - 1), 2: (-360, 720), 3: (1, 89), 4: (-200, 200), 5: (1, 600),
              6: (0.05, 30), 7: (1, 300), 8: (0.1, 5), 9: (0.05, 5)}
    for k in free:
        lo[k], hi[k] = bounds[k]
    p0 = np.array([synth.perturb(rng, truth, free, frac, lo, hi) for _ in range(6)])
    opts = G.lm_opts(max_iter=200, free=free, jacobian=jacobian if jacobian is not None else G.JAC_FD_FORWARD)
    q, c, it, st = G.fit_lm(g, [d] * 6, p0, [lo] * 6, [hi] * 6, opts)
    return truth, q, c, it, st


@pytest.mark.parametrize("model", [VF_ARCTAN, VF_EPINAT])
def test_vfield_tangent_fit_recovers(G, model):
    """LM with the analytic velocity-field Jacobian recovers the truth from
    perturbed starts (20 % arctan, 5 % Epinat) like the FD LM does."""
    truth, q, c, it, st = _fit_case(G, model, 9, 0.2 if model == VF_ARCTAN else 0.05, G.JAC_TANGENT)
    assert np.all(np.isin(st, [1, 2])), (st, it)
    assert np.all(c < 1e-3), c
    assert np.all(np.abs(q[:, 2] - truth[2]) < 1.0), q[:, 2]
    assert np.all(np.abs(q[:, 5] - truth[5]) < 2.0), q[:, 5]


def test_vfield_arctan_fit_recovers(G):
    truth, q, c, it, st = _fit_case(G, VF_ARCTAN, 7, 0.2)
    assert np.all(np.isin(st, [1, 2])), (st, it)
    assert np.all(np.abs(q[:, 5] - truth[5]) < 2.0), q[:, 5]
    assert np.all(np.abs(q[:, 2] - truth[2]) < 1.0), q[:, 2]


def test_vfield_epinat_fit_recovers(G):
    """The nine-parameter GHASP problem (Sec. 4.2: velocity field, Epinat
    curve): noiseless field from 5 %-perturbed starts."""
    truth, q, c, it, st = _fit_case(G, VF_EPINAT, 8, 0.05)
    assert np.all(np.isin(st, [1, 2])), (st, it)
    assert np.all(c < 1e-3), c
    assert np.all(np.abs(q[:, 2] - truth[2]) < 1.0), q[:, 2]
    assert np.all(np.abs(q[:, 3] - truth[3]) < 2.0), q[:, 3]


def test_vfield_grid_argmin_matches_oracle(G):
    g = vgeom(40, 40, VF_EPINAT)
    truth = np.array([19.5, 20.2, 60.0, 45.0, 0.0, 180.0, 5.0, 30.0, 1.2, 0.8])
    m = oracle.evaluate(ogeom(g), truth)
    wv, ws = synth.weights((40, 40), 5.0)
    ob = oracle.Obs(m[1].astype(np.float32), m[2].astype(np.float32), wv, ws, np.ones((40, 40), np.uint8))
    lo, hi = truth.copy(), truth.copy()
    nodes = [1] * 10
    for k, (a, b, n) in {2: (30.0, 90.0, 7), 5: (120.0, 240.0, 7), 8: (0.4, 2.0, 5), 9: (0.4, 1.2, 5)}.items():
        lo[k], hi[k], nodes[k] = a, b, n
    bp, bi, bc, _ = fit.grid_search(ogeom(g), ob, lo, hi, nodes, truth, levels=2)
    d = G.Obs.from_numpy(ob.v, ob.s, ob.w_v, ob.w_s, ob.mask)
    gp, gi, gc = G.gbk_grid(g, d, lo, hi, nodes, truth, levels=2, chunk=512)
    assert list(gi) == list(bi), (gi, bi)
