"""gbk_chi2_host: the split evaluator called with parameters, observed maps
and chi2 in host memory.  The maps' copy runs on the PSF stages' stream,
beside the first line stage; the result must equal gbk_chi2 on device
copies of the same inputs bit for bit, for one chunk and for several, from
pinned and from pageable host memory, and for calls back to back on one
workspace."""
import numpy as np
import pytest
import torch

from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def _host_obs(G, g, p, seed, pin):
    maps = G.eval_maps(g, torch.from_numpy(p[None]))[0].cpu().numpy()
    rng = np.random.default_rng(seed)
    shape = (g.ny, g.nx)
    v = (maps[1] + rng.normal(0, 5.0, shape)).astype(np.float32)
    s = (maps[2] + rng.normal(0, 5.0 * np.sqrt(2.0), shape)).astype(np.float32)
    wv, ws = synth.weights(shape, 5.0)
    mask = synth.dead_fibre_mask(rng, shape).astype(np.uint8)
    t = [torch.from_numpy(np.ascontiguousarray(a)) for a in (v, s, wv.astype(np.float32), ws.astype(np.float32), mask)]
    if pin:
        t = [a.pin_memory() for a in t]
    return G.Obs(*t)


@pytest.mark.parametrize("n,pin", [(400, True), (37, True), (400, False)])
def test_host_call_equals_device_call(G, n, pin):
    g = synth.FP_GEOM
    rng = np.random.default_rng(n)
    p = synth.draw_fp_params(rng, n)
    h_obs = _host_obs(G, g, p[0], 9, pin)
    d_obs = G.Obs(*[a.cuda() for a in (h_obs.v_obs, h_obs.s_obs, h_obs.w_v, h_obs.w_s, h_obs.mask)])
    want = torch.empty(n, dtype=torch.float64, device="cuda")
    ws_dev = torch.empty(G.gbk_workspace_bytes(g, n, G.PATH_SPLIT), dtype=torch.uint8, device="cuda")
    G.gbk_chi2(g, torch.from_numpy(p).cuda(), d_obs, want, None, G.PATH_SPLIT, ws_dev)
    h_p = torch.from_numpy(p)
    h_chi2 = torch.full((n,), -1.0, dtype=torch.float64)
    if pin:
        h_p, h_chi2 = h_p.pin_memory(), h_chi2.pin_memory()
    ws = torch.empty(G.gbk_chi2_host_workspace_bytes(g, n), dtype=torch.uint8, device="cuda")
    G.gbk_chi2_host(g, h_p, h_obs, h_chi2, ws)
    torch.cuda.synchronize()
    assert torch.equal(h_chi2, want.cpu())
    # back to back on the same workspace with other parameters: the second
    # call's copies wait for the first call's stages
    p2 = synth.draw_fp_params(rng, n)
    h_p2 = torch.from_numpy(p2)
    h_chi2b = torch.full((n,), -1.0, dtype=torch.float64)
    if pin:
        h_p2, h_chi2b = h_p2.pin_memory(), h_chi2b.pin_memory()
    G.gbk_chi2_host(g, h_p, h_obs, h_chi2, ws)
    G.gbk_chi2_host(g, h_p2, h_obs, h_chi2b, ws)
    G.gbk_chi2(g, torch.from_numpy(p2).cuda(), d_obs, want, None, G.PATH_SPLIT, ws_dev)
    torch.cuda.synchronize()
    assert torch.equal(h_chi2b, want.cpu())


def test_host_call_rejects_what_the_split_path_does_not_serve(G):
    g = synth.FP_GEOM.with_(upsample=2)
    with pytest.raises(G.GbkError):
        G.gbk_chi2_host_workspace_bytes(g, 4)
