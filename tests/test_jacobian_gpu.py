"""The analytic Jacobian kernel (gbk_jacobian) against central differences of
the FP64 oracle, its J^T J / J^T r reductions, the torch.autograd wrapper and
LM driven by it."""
import numpy as np
import pytest
import torch

import oracle
from oracle import fit
from cases import ogeom, make_obs, model_params
from lm_cases import FREE, bounds, galaxy, starts
from paper_1510_01815_gb300 import synth
from paper_1510_01815_gb300.synth import Geometry, params as P

pytestmark = pytest.mark.gpu

# central-difference steps of the oracle (FP64), per parameter
STEPS = np.array([1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-3, 1e-4, 1e-3, 1e-5, 1e-4])


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def oracle_jacobian(g, p, obs):
    og = ogeom(g)
    cols = []
    for k in range(10):
        a, b = p.copy(), p.copy()
        a[k] += STEPS[k]
        b[k] -= STEPS[k]
        _, r = oracle.chi2_batch(og, np.array([a, b]), obs, want_resid=True)
        cols.append((r[0] - r[1]) / (2 * STEPS[k]))
    return np.array(cols)  # [10][2][ny][nx]


CASES = {
    "single": (synth.SINGLE_GEOM, synth.SINGLE_TRUTH),
    "single_mode1": (synth.SINGLE_GEOM.with_(lsf_mode=1), synth.SINGLE_TRUTH),
    "nonsquare": (Geometry(40, 24, 32, 15.0, 0.0, 2.0, 35.0), P(19.7, 12.2, 145, 58, 0, 210, 3, 35, 1, 5)),
    "narrow_band": (Geometry(9, 7, 4, 10.0, 0.0, 2.0, 60.0), P(4.1, 3.2, 10, 40, 0, 30, 2, 20, 1, 3)),
    # too wide for halo copies in shared memory: the y pass reads the halo
    # rows in the neighbouring CTAs' shared memory
    "direct_halo": (Geometry(72, 72, 40, 20.0, 0.0, 4.0, 30.0), P(35.2, 36.1, 30, 55, 0, 180, 5, 40, 1, 9)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_jacobian_matches_central_differences(G, case):
    g, p = CASES[case]
    ps = model_params(g, p, 3, seed=13)
    obs = make_obs(g, p, seed=3)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    jac, jtj, jtv, c2 = G.jacobian(g, torch.from_numpy(ps), dobs, free=tuple(range(10)))
    jac = jac.cpu().numpy()
    for i in range(ps.shape[0]):
        ref = oracle_jacobian(g, ps[i], obs)
        overall = np.abs(ref).max()
        for k in range(10):
            # a column that vanishes (the maps do not depend on I0) is judged
            # against the Jacobian's overall scale
            scale = max(np.abs(ref[k]).max(), 1e-3 * overall)
            err = np.abs(jac[i, k] - ref[k]).max() / scale
            assert err < 3e-3, (case, i, synth.PARAM_NAMES[k], err)


def test_reductions_match_own_jacobian(G):
    g, p = synth.SINGLE_GEOM, synth.SINGLE_TRUTH
    ps = model_params(g, p, 4, seed=14)
    obs = make_obs(g, p, seed=6)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    jac, jtj, jtv, c2 = G.jacobian(g, torch.from_numpy(ps), dobs, free=FREE)
    _, r = oracle.chi2_batch(ogeom(g), ps, obs, want_resid=True)
    ref_c = oracle.chi2_batch(ogeom(g), ps, obs)
    jac = jac.cpu().numpy().astype(np.float64)
    for i in range(ps.shape[0]):
        J = jac[i][list(FREE)].reshape(len(FREE), -1).T
        np.testing.assert_allclose(jtj[i].cpu().numpy(), J.T @ J, rtol=1e-4, atol=1e-6 * np.abs(J.T @ J).max())
        g_ref = J.T @ r[i].ravel()
        np.testing.assert_allclose(jtv[i].cpu().numpy(), g_ref, rtol=2e-3, atol=2e-3 * np.abs(g_ref).max())
        assert abs(c2[i].item() - ref_c[i]) < 1e-3 * ref_c[i]


def test_autograd_wrapper(G):
    """grad of 0.5 * sum(resid^2) through ResidualMaps equals J^T r."""
    g, p = synth.SINGLE_GEOM, synth.SINGLE_TRUTH
    ps = model_params(g, p, 2, seed=15)
    obs = make_obs(g, p, seed=7)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    x = torch.from_numpy(ps).cuda().requires_grad_(True)
    res = G.residual_maps(x, g, dobs)
    loss = 0.5 * (res.double() ** 2).sum()
    loss.backward()
    jac, jtj, jtv, c2 = G.jacobian(g, torch.from_numpy(ps), dobs, free=tuple(range(10)))
    # the backward pass uses the fused kernel's residuals as cotangent, jtv
    # the tangent kernel's own: they agree to FP32 rounding of the maps
    ref_g = jtv.cpu().numpy()
    np.testing.assert_allclose(x.grad.cpu().numpy(), ref_g, rtol=0, atol=1e-4 * np.abs(ref_g).max())
    # and against the oracle's central-difference gradient of chi2 / 2
    ref = oracle_jacobian(g, ps[0], obs)
    _, r = oracle.chi2_batch(ogeom(g), ps[:1], obs, want_resid=True)
    gref = np.einsum("kij,ij->k", ref.reshape(10, 2, -1).reshape(10, 2, g.ny * g.nx), r[0].reshape(2, -1))
    sc = np.abs(gref).max()
    assert np.all(np.abs(x.grad[0].cpu().numpy() - gref) <= 3e-3 * sc), (x.grad[0].cpu().numpy(), gref)


def test_lm_with_tangent_jacobian(G):
    """Noiseless recovery (Sec. 4.1 thresholds) and, on noisy data, the same
    chi2 minimum as the finite-difference LM."""
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    n = 8
    p0 = starts(p, n, seed=31)
    d = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    opts = G.lm_opts(max_iter=100, jacobian=G.JAC_TANGENT, free=FREE)
    q, c, it, st = G.fit_lm(g, [d] * n, p0, [lo] * n, [hi] * n, opts)
    assert np.all(np.isin(st, [1, 2])), (st, it)
    assert np.all(np.abs(q[:, synth.VMAX] - p[synth.VMAX]) < 2.0)
    assert np.all(np.abs(q[:, synth.PA] - p[synth.PA]) < 1.0)
    g, p, obs = galaxy(noise_v=5.0, seed=4)
    d = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    p0 = starts(p, 1, seed=9)
    qt, ct, _, _ = G.fit_lm(g, [d], p0, lo[None], hi[None], opts)
    qf, cf, _, _ = G.fit_lm(g, [d], p0, lo[None], hi[None], G.lm_opts(max_iter=100, free=FREE))
    assert ct[0] <= cf[0] * (1 + 1e-4), (ct, cf)


# The split-shape Jacobian (gbk_jacobian_ws): the same reductions as the
# cluster kernel, whose J is checked above element by element against
# central differences of the oracle, and against J^T J and J^T r formed from
# the oracle's central-difference J directly.  Both kernels carry FP32
# derivative triplets through the same arithmetic up to the order and form
# of the PSF accumulation, so they agree to a few 1e-4 of the largest entry.
SPLIT_CASES = ["single", "single_mode1", "nonsquare", "narrow_band", "direct_halo"]


def _split_vs_cluster(G, g, ps, dobs, free, cot=None):
    n, nf = ps.shape[0], len(free)
    par = torch.from_numpy(ps).cuda()
    out = {}
    for name in ("cluster", "split"):
        jtj = torch.empty((n, nf, nf), dtype=torch.float64, device="cuda")
        jtv = torch.empty((n, nf), dtype=torch.float64, device="cuda")
        c2 = torch.empty(n, dtype=torch.float64, device="cuda")
        if name == "cluster":
            G.gbk_jacobian(g, par, dobs, free, cot, jtj, jtv, c2, None)
        else:
            ws = torch.empty(G.gbk_jacobian_workspace_bytes(g, n, free), dtype=torch.uint8, device="cuda")
            G.gbk_jacobian_ws(g, par, dobs, free, cot, jtj, jtv, c2, ws)
        torch.cuda.synchronize()
        out[name] = (jtj.cpu().numpy(), jtv.cpu().numpy(), c2.cpu().numpy())
    return out["cluster"], out["split"]


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_split_jacobian_matches_cluster_kernel_and_oracle(G, case):
    g, p = CASES[case]
    ps = model_params(g, p, 3, seed=17)
    obs = make_obs(g, p, seed=3)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    (a_jtj, a_jtv, a_c), (b_jtj, b_jtv, b_c) = _split_vs_cluster(G, g, ps, dobs, FREE)
    for i in range(ps.shape[0]):
        s = np.abs(a_jtj[i]).max()
        assert np.abs(b_jtj[i] - a_jtj[i]).max() <= 1e-3 * s, (case, i, np.abs(b_jtj[i] - a_jtj[i]).max() / s)
        sv = np.abs(a_jtv[i]).max()
        assert np.abs(b_jtv[i] - a_jtv[i]).max() <= 1e-3 * sv, (case, i)
        assert abs(b_c[i] - a_c[i]) <= 1e-4 * a_c[i] + 1e-9, (case, i, b_c[i], a_c[i])
    # against the oracle's central-difference Jacobian
    _, r = oracle.chi2_batch(ogeom(g), ps, obs, want_resid=True)
    for i in range(ps.shape[0]):
        J = oracle_jacobian(g, ps[i], obs)[list(FREE)].reshape(len(FREE), -1).T
        ref = J.T @ J
        assert np.abs(b_jtj[i] - ref).max() <= 1e-2 * np.abs(ref).max(), (case, i)
        gref = J.T @ r[i].ravel()
        assert np.abs(b_jtv[i] - gref).max() <= 1e-2 * np.abs(gref).max(), (case, i)


def test_split_jacobian_in_chunks_with_cotangent(G):
    """More models than one L2-sized chunk (334 at 32 x 32), a
    cotangent in place of the residuals, and fewer free parameters: the
    output keeps the order of the free parameters."""
    g, p = synth.SINGLE_GEOM, synth.SINGLE_TRUTH
    n = 700
    ps = model_params(g, p, n, seed=18)
    obs = make_obs(g, p, seed=5)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    rng = np.random.default_rng(19)
    cot = torch.from_numpy(rng.normal(size=(n, 2, g.ny, g.nx)).astype(np.float32)).cuda()
    free = (synth.PA, synth.VMAX, synth.X0, synth.SIG0)
    (a_jtj, a_jtv, a_c), (b_jtj, b_jtv, b_c) = _split_vs_cluster(G, g, ps, dobs, free, cot)
    for i in (0, 1, 333, 334, 667, 668, n - 1):
        s = np.abs(a_jtj[i]).max()
        assert np.abs(b_jtj[i] - a_jtj[i]).max() <= 1e-3 * s, i
        assert np.abs(b_jtv[i] - a_jtv[i]).max() <= 1e-3 * np.abs(a_jtv[i]).max(), i
    np.testing.assert_allclose(b_c, a_c, rtol=1e-4)


def test_split_jacobian_refuses_what_it_does_not_serve(G):
    g = synth.SINGLE_GEOM
    with pytest.raises(G.GbkError):  # I0 and h are not carried
        G.gbk_jacobian_workspace_bytes(g, 4, tuple(range(10)))
    with pytest.raises(G.GbkError):  # PSF radius 16 > 8
        G.gbk_jacobian_workspace_bytes(g.with_(psf_fwhm=9.0), 4, FREE)
    ps = model_params(g, synth.SINGLE_TRUTH, 4, seed=20)
    obs = make_obs(g, synth.SINGLE_TRUTH, seed=5)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    jtj = torch.full((4, 8, 8), -1.0, dtype=torch.float64, device="cuda")
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(G.GbkError) as ei:
        G.gbk_jacobian_ws(g, torch.from_numpy(ps).cuda(), dobs, FREE, None, jtj, None, None, small)
    assert ei.value.status == G.GBK_EWORKSPACE
    torch.cuda.synchronize()
    assert torch.all(jtj == -1.0)
