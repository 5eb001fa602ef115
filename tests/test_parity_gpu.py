"""GPU parity: the CUDA forward model against the FP64 oracle, element by
element, through the C ABI.  Tolerances are stated in tests/cases.py."""
import numpy as np
import pytest
import torch

import oracle
from cases import ogeom, make_obs, model_params, check_maps, chi2_bound
from paper_1510_01815_gb300 import synth
from paper_1510_01815_gb300.synth import Geometry, params as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    return gbk


CASES = {
    "single": (synth.SINGLE_GEOM, synth.SINGLE_TRUTH),
    "single_mode1": (synth.SINGLE_GEOM.with_(lsf_mode=1), synth.SINGLE_TRUTH),
    "no_conv": (synth.SINGLE_GEOM.with_(psf_fwhm=0.0, lsf_fwhm=0.0), synth.SINGLE_TRUTH),
    "tiny_1x1x1": (Geometry(1, 1, 1, 20.0, 0.0, 2.5, 30.0), P(0.3, 0.2, 40, 50, 0, 150, 2, 40, 1, 3)),
    "odd_3x5x7": (Geometry(3, 5, 7, 40.0, 0.0, 1.5, 50.0), P(1.2, 2.3, 200, 35, 10, 120, 1.5, 30, 2, 2)),
    "prime_13x11x17": (Geometry(13, 11, 17, 25.0, 0.0, 3.3, 45.0), P(6.4, 4.9, 75, 62, -5, 180, 2.5, 25, 1, 3)),
    "narrow_band": (Geometry(9, 7, 4, 10.0, 0.0, 2.0, 60.0), P(4.1, 3.2, 10, 40, 0, 30, 2, 20, 1, 3)),
    "wide_kernels": (Geometry(24, 20, 40, 10.0, 5.0, 9.0, 150.0), P(11.6, 9.3, 300, 45, 5, 90, 4, 30, 1, 6)),
    "grid64": (synth.GRID_GEOM, P(33.1, 30.7, 222, 48, 0, 240, 5.5, 55, 1, 12)),
    "nonsquare": (Geometry(40, 24, 32, 15.0, 0.0, 2.0, 35.0), P(19.7, 12.2, 145, 58, 0, 210, 3, 35, 1, 5)),
    "edge_on": (synth.SINGLE_GEOM, P(15.5, 15.5, 120, 88.5, 0, 200, 3, 40, 1, 1.0)),
    "vc_offset": (synth.SINGLE_GEOM.with_(vc=100.0), P(15.2, 16.1, 30, 50, 100, 200, 3, 40, 1, 4)),
    # every line centred 7-7.5 sigma beyond the last extended channel (690
    # km/s): each spaxel's in-band flux is its Gaussian tail at |u| in
    # (6, 11.25), 1e-20 .. 7e-17 of I0 -- valid spectra (above the 1e-20 I0
    # threshold) that a channel window cut at |u| = 6 would empty
    "line_beyond_band": (synth.SINGLE_GEOM, P(15.5, 15.5, 120, 55, 988.8, 10, 3, 40, 1, 4)),
}


def _params(case, n=4, seed=7):
    g, p = CASES[case]
    ps = model_params(g, p, n, seed)
    ps[:, synth.INCL] = np.minimum(ps[:, synth.INCL], 89.0)
    return g, p, ps


@pytest.mark.parametrize("case", sorted(CASES))
def test_maps_fused_vs_oracle(G, case):
    g, p, ps = _params(case)
    ref = oracle.evaluate_batch(ogeom(g), ps)
    maps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    check_maps(maps, ref, ps, case)
    if case == "line_beyond_band":  # the case has the valid tail spectra it is meant to have
        assert (ref[0, 0] >= 2e-20).sum() > 900 and ref[0, 0].max() < 1e-16


# The split path (two stages meeting in an L2-resident buffer of moment
# triplets) serves PSF radii up to 8 px: every case but wide_kernels.
SPLIT_CASES = [c for c in sorted(CASES) if c != "wide_kernels"]


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_maps_split_vs_oracle(G, case):
    g, p, ps = _params(case)
    ref = oracle.evaluate_batch(ogeom(g), ps)
    maps = G.eval_maps(g, torch.from_numpy(ps), split=True).cpu().numpy()
    check_maps(maps, ref, ps, case + " (split)")
    # the fused path's arithmetic, spaxels grouped into warps differently:
    # the sums differ only by terms below 2^-36 of the line peak and by FP32
    # rounding, so the maps agree far inside the oracle tolerance
    fused = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    for k in range(3):
        scale = np.nanmax(np.abs(fused[:, k])) if np.isfinite(fused[:, k]).any() else 1.0
        np.testing.assert_allclose(maps[:, k], fused[:, k], rtol=1e-5, atol=1e-6 * scale)


def test_split_refuses_wide_kernels(G):
    g, p, ps = _params("wide_kernels")
    assert G.gbk_workspace_bytes(g, 4, G.PATH_SPLIT) == 0
    obs = make_obs(g, p, seed=3)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GbkError) as ei:
        G.gbk_chi2(g, torch.from_numpy(ps).cuda(), dobs, out, None, G.PATH_SPLIT, None)
    assert ei.value.status == G.GBK_EUNSUPPORTED
    # the automatic choice falls back to the fused path
    c = G.chi2(g, torch.from_numpy(ps), dobs).cpu().numpy()
    np.testing.assert_allclose(c, oracle.chi2_batch(ogeom(g), ps, obs), rtol=1e-3)


def test_split_needs_its_workspace(G):
    g, p, ps = _params("single")
    obs = make_obs(g, p, seed=3)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    need = G.gbk_workspace_bytes(g, 4, G.PATH_SPLIT)
    assert need > 0 and G.gbk_workspace_bytes(g, 4, G.PATH_AUTO) == need
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GbkError) as ei:
        G.gbk_chi2(g, torch.from_numpy(ps).cuda(), dobs, out, None, G.PATH_SPLIT, small)
    assert ei.value.status == G.GBK_EWORKSPACE
    # AUTO with too small a workspace (or none) takes the fused path
    G.gbk_chi2(g, torch.from_numpy(ps).cuda(), dobs, out, None, G.PATH_AUTO, small)
    ref = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_FUSED)
    assert torch.equal(out, ref)


@pytest.mark.parametrize("case", ["single", "single_mode1", "tiny_1x1x1", "odd_3x5x7", "narrow_band",
                                  "wide_kernels", "nonsquare", "edge_on", "line_beyond_band"])
def test_cube_and_maps_staged_vs_oracle(G, case):
    g, p, ps = _params(case, n=3)
    cubes, maps = G.eval_cubes(g, torch.from_numpy(ps))
    assert G.gbk_device_status() == 0
    cubes, maps = cubes.cpu().numpy(), maps.cpu().numpy()
    for i in range(ps.shape[0]):
        cref, mref = oracle.evaluate(ogeom(g), ps[i], want_cube=True)
        scale = np.abs(cref).max()
        err = np.abs(cubes[i] - cref).max() / scale
        assert err <= 1e-4, "%s model %d cube rel err %.3g" % (case, i, err)
        check_maps(maps[i:i + 1], mref[None], ps[i:i + 1], case)


@pytest.mark.parametrize("u,case", [(2, "single"), (2, "odd_3x5x7"), (3, "tiny_1x1x1"), (2, "nonsquare")])
def test_upsampled_staged_vs_oracle(G, u, case):
    g, p, ps = _params(case, n=2)
    g = g.with_(upsample=u)
    ref = oracle.evaluate_batch(ogeom(g), ps)
    maps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    check_maps(maps, ref, ps, "%s u=%d" % (case, u))
    cubes, maps2 = G.eval_cubes(g, torch.from_numpy(ps))
    cref, _ = oracle.evaluate(ogeom(g), ps[0], want_cube=True)
    assert np.abs(cubes[0].cpu().numpy() - cref).max() <= 1e-4 * np.abs(cref).max()


@pytest.mark.parametrize("case", ["single", "single_mode1", "grid64", "nonsquare", "edge_on", "prime_13x11x17"])
@pytest.mark.parametrize("path", ["fused", "staged", "split"])
def test_chi2_vs_oracle(G, case, path):
    g, p, ps = _params(case, n=5, seed=11)
    obs = make_obs(g, p, seed=3)
    flags = {"fused": G.PATH_FUSED, "staged": G.PATH_STAGED, "split": G.PATH_SPLIT}[path]
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    c, resid = G.chi2(g, torch.from_numpy(ps), dobs, flags=flags, want_resid=True)
    c, resid = c.cpu().numpy(), resid.cpu().numpy()
    ref_c, ref_r = oracle.chi2_batch(ogeom(g), ps, obs, want_resid=True)
    if path == "fused":
        gmaps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    elif path == "split":
        gmaps = G.eval_maps(g, torch.from_numpy(ps), split=True).cpu().numpy()
    else:
        gmaps = G.eval_cubes(g, torch.from_numpy(ps))[1].cpu().numpy()
    rmaps = oracle.evaluate_batch(ogeom(g), ps)
    for i in range(ps.shape[0]):
        bound = chi2_bound(rmaps[i], gmaps[i], obs, ref_c[i])
        assert abs(c[i] - ref_c[i]) <= bound, (case, path, i, c[i], ref_c[i], bound)
        # residual maps: same bound per spaxel from the map deviation
        dv = np.abs(obs.w_v * (gmaps[i][1] - rmaps[i][1]))
        ds = np.abs(obs.w_s * (gmaps[i][2] - rmaps[i][2]))
        use = (obs.mask != 0) & (rmaps[i][0] > 0)
        assert np.all(np.abs(resid[i][0] - ref_r[i][0])[use] <= dv[use] + 1e-5 * np.abs(ref_r[i][0][use]) + 1e-6)
        assert np.all(np.abs(resid[i][1] - ref_r[i][1])[use] <= ds[use] + 1e-5 * np.abs(ref_r[i][1][use]) + 1e-6)
        assert np.all(resid[i][:, obs.mask == 0] == 0)


@pytest.mark.parametrize("u", [1, 2])
def test_stage_times_run_the_staged_chi2(G, u):
    """gbk_chi2_stage_times computes exactly gbk_chi2 on the staged path and
    times its stages; the down-sampling stage is empty at u = 1."""
    g, p, ps = _params("nonsquare", n=4, seed=5)
    g = g.with_(upsample=u)
    obs = make_obs(g.with_(upsample=1), p, seed=3)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    par = torch.from_numpy(ps).cuda()
    ws = G.workspace_for(g, ps.shape[0], G.PATH_STAGED, "cuda")
    c0 = torch.empty(ps.shape[0], dtype=torch.float64, device="cuda")
    c1 = torch.empty_like(c0)
    G.gbk_chi2(g, par, dobs, c0, None, G.PATH_STAGED, ws)
    ms = G.gbk_chi2_stage_times(g, par, dobs, c1, ws)
    assert torch.equal(c0, c1)
    assert len(ms) == 4 and all(t >= 0.0 for t in ms)
    assert ms[0] > 0.0 and ms[1] > 0.0 and ms[3] > 0.0
    if u == 1:
        assert ms[2] < 0.02  # back-to-back events: a few microseconds
    else:
        assert ms[2] > 0.0


def test_chi2_reduction_on_identical_maps(G):
    """The reduction alone, on the same FP32 maps: 1e-5 relative."""
    g = synth.SINGLE_GEOM
    ps = model_params(g, synth.SINGLE_TRUTH, 6, seed=5)
    maps = oracle.evaluate_batch(ogeom(g), ps).astype(np.float32)
    obs = make_obs(g, synth.SINGLE_TRUTH, seed=4)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    resid = torch.empty((6, 2, g.ny, g.nx), dtype=torch.float32, device="cuda")
    G.gbk_chi2_from_maps(torch.from_numpy(maps).cuda(), dobs, out, resid)
    torch.cuda.synchronize()
    for i in range(6):
        ref, rr = oracle.chi2_maps(maps[i].astype(np.float64), obs, want_resid=True)
        assert abs(out[i].item() - ref) <= 1e-5 * ref + 1e-12, (i, out[i].item(), ref)
        np.testing.assert_allclose(resid[i].cpu().numpy(), rr, rtol=1e-5, atol=1e-6)


def test_noiseless_truth_gives_zero_chi2(G):
    """Observed maps made by the same GPU path at the same parameters: chi2 = 0
    exactly (bitwise-identical maps)."""
    g, p = synth.SINGLE_GEOM, synth.SINGLE_TRUTH
    maps = G.eval_maps(g, torch.from_numpy(p[None]))
    wv, ws = synth.weights((g.ny, g.nx), 5.0)
    dobs = G.Obs(maps[0, 1].contiguous(), maps[0, 2].contiguous(), torch.from_numpy(wv).cuda(),
                 torch.from_numpy(ws).cuda(), torch.ones((g.ny, g.nx), dtype=torch.uint8, device="cuda"))
    c = G.chi2(g, torch.from_numpy(p[None]), dobs, flags=G.PATH_FUSED)
    assert c.item() == 0.0


def test_bitwise_deterministic(G):
    g, p, ps = _params("grid64", n=8)
    obs = make_obs(g, p, seed=9)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    a = G.chi2(g, torch.from_numpy(ps), dobs).cpu().numpy()
    b = G.chi2(g, torch.from_numpy(ps), dobs).cpu().numpy()
    assert np.array_equal(a, b)
    m1 = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    m2 = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    assert np.array_equal(m1, m2)


def test_invalid_parameters_give_nan(G):
    g = synth.SINGLE_GEOM
    ps = np.array([synth.SINGLE_TRUTH] * 4)
    ps[1, synth.INCL] = 90.0
    ps[2, synth.SIG0] = -1.0
    ps[3, synth.RT] = np.nan
    obs = make_obs(g, synth.SINGLE_TRUTH, seed=1)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    ref = oracle.chi2_batch(ogeom(g), ps, obs)  # the same parameter domain on both sides
    for flags in (G.PATH_FUSED, G.PATH_STAGED, G.PATH_SPLIT):
        c = G.chi2(g, torch.from_numpy(ps), dobs, flags=flags).cpu().numpy()
        assert np.isfinite(c[0]) and np.all(np.isnan(c[1:])), (flags, c)
        assert np.array_equal(np.isnan(c), np.isnan(ref)), (flags, c, ref)
    for split in (False, True):
        maps = G.eval_maps(g, torch.from_numpy(ps), split=split).cpu().numpy()
        assert np.isfinite(maps[0]).all() and np.isnan(maps[1:]).all()
        assert np.array_equal(np.isnan(maps), np.isnan(oracle.evaluate_batch(ogeom(g), ps)))


def test_fused_and_staged_agree(G):
    g, p, ps = _params("nonsquare", n=6)
    obs = make_obs(g, p, seed=2)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    a = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_FUSED).cpu().numpy()
    b = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_STAGED).cpu().numpy()
    np.testing.assert_allclose(a, b, rtol=2e-4)


@pytest.mark.slow
def test_fabry_perot_split_in_chunks(G):
    """192 x 192 x 48, 150 models: more than one L2-sized chunk of the split
    path (80 models each), each chunk's chi2 and maps against the fused
    path and sampled models against the oracle, in the batch the benchmark
    times (400 models) as well."""
    g = synth.FP_GEOM
    rng = np.random.default_rng(23)
    for n in (150, 400):
        ps = synth.draw_fp_params(rng, n)
        p_true = ps[0]
        m_true = oracle.evaluate(ogeom(g), p_true)
        shape = (g.ny, g.nx)
        obs = oracle.Obs((m_true[1] + rng.normal(0, 5, shape)).astype(np.float32),
                         (m_true[2] + rng.normal(0, 7.07, shape)).astype(np.float32),
                         *synth.weights(shape, 5.0),
                         (synth.sn_mask(m_true[0]) * synth.dead_fibre_mask(rng, shape)).astype(np.uint8))
        dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
        cs = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_SPLIT).cpu().numpy()
        cf = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_FUSED).cpu().numpy()
        np.testing.assert_allclose(cs, cf, rtol=1e-5)
        ms = G.eval_maps(g, torch.from_numpy(ps), split=True).cpu().numpy()
        for i in (0, 79, 80, n - 1):
            rm = oracle.evaluate(ogeom(g), ps[i])
            check_maps(ms[i:i + 1], rm[None], ps[i:i + 1], "fp split model %d of %d" % (i, n))
            rc = oracle.chi2_maps(rm, obs)
            assert abs(cs[i] - rc) <= chi2_bound(rm, ms[i], obs, rc), (i, cs[i], rc)


@pytest.mark.slow
def test_fabry_perot_full_size(G):
    """192 x 192 x 48 at the launch configuration the benchmark times (a
    cluster of CTAs per model), full maps of two models against the oracle and
    chi2 of a 400-model batch against sampled oracle models."""
    g = synth.FP_GEOM
    rng = np.random.default_rng(21)
    ps = synth.draw_fp_params(rng, 400)
    ref = oracle.evaluate_batch(ogeom(g), ps[:2])
    maps = G.eval_maps(g, torch.from_numpy(ps[:2])).cpu().numpy()
    check_maps(maps, ref, ps[:2], "fp")
    p_true = ps[0]
    m_true = ref[0]
    shape = (g.ny, g.nx)
    obs = oracle.Obs((m_true[1] + rng.normal(0, 5, shape)).astype(np.float32),
                     (m_true[2] + rng.normal(0, 7.07, shape)).astype(np.float32),
                     *synth.weights(shape, 5.0),
                     (synth.sn_mask(m_true[0]) * synth.dead_fibre_mask(rng, shape)).astype(np.uint8))
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    c = G.chi2(g, torch.from_numpy(ps), dobs).cpu().numpy()
    allmaps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    for i in (0, 1, 137, 399):
        rm = ref[i] if i < 2 else oracle.evaluate(ogeom(g), ps[i])
        rc = oracle.chi2_maps(rm, obs)
        assert abs(c[i] - rc) <= chi2_bound(rm, allmaps[i], obs, rc), (i, c[i], rc)


@pytest.mark.parametrize("case,cs,threads,pers", [
    ("grid64", 1, 512, 0), ("grid64", 2, 384, 1), ("grid64", 3, 256, 0), ("grid64", 5, 512, 1),
    ("grid64", 16, 384, 0), ("single", 1, 256, 1), ("single", 7, 512, 0), ("nonsquare", 4, 384, 1),
    ("wide_kernels", 6, 512, 0), ("prime_13x11x17", 16, 256, 1)])
def test_every_tuning_matches_oracle(G, case, cs, threads, pers):
    """Forced launch configurations (CTAs per model, block size, grid shape)
    all give the oracle's maps; chi2 of all 600 models agrees with the
    default configuration (a persistent grid loops several models per
    cluster at this batch size)."""
    g, p, ps = _params(case, n=600)
    sample = [0, 1, 299, 598, 599]
    ref = oracle.evaluate_batch(ogeom(g), ps[sample])
    obs = make_obs(g, p, seed=5)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    base = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_FUSED).cpu().numpy()
    try:
        G.gbk_set_tuning(g, cs, threads, pers)
        maps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
        c = G.chi2(g, torch.from_numpy(ps), dobs, flags=G.PATH_FUSED).cpu().numpy()
    finally:
        G.gbk_set_tuning(g, None)
    check_maps(maps[sample], ref, ps[sample], "%s cs=%d nt=%d pers=%d" % (case, cs, threads, pers))
    np.testing.assert_allclose(c, base, rtol=1e-5)


def test_autotune_picks_a_valid_tuning(G):
    g, p, ps = _params("grid64", n=16)
    obs = make_obs(g, p, seed=6)
    dobs = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    scratch = torch.empty(16, dtype=torch.float64, device="cuda")
    try:
        t = G.gbk_autotune(g, torch.from_numpy(ps).cuda(), dobs, scratch)
        assert t["candidates"] >= 3 and t["ms"] > 0
        assert G.gbk_get_tuning(g) == {"cluster_ctas": t["cluster_ctas"], "threads": t["threads"],
                                       "persistent": t["persistent"]}
        maps = G.eval_maps(g, torch.from_numpy(ps)).cpu().numpy()
    finally:
        G.gbk_set_tuning(g, None)
    check_maps(maps, oracle.evaluate_batch(ogeom(g), ps), ps, "autotuned")
