"""gbk_chi2_noalloc: the staged chi-squared path with the library's built-in
scratch, for callers that cannot allocate device memory (for example a
plug-in whose host framework owns all device memory).  Its results must
equal those of gbk_chi2 with a caller workspace bit for bit on calls in a
row (across two layouts), and oversized batches must be refused before
anything runs.  This file is collected last so a stop at its first failure
has already run the others."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available(), "the -m gpu tests need a CUDA device"
    return gbk


def _obs(G, g, seed):
    rng = np.random.default_rng(seed)
    shape = (g.ny, g.nx)
    truth = synth.SINGLE_TRUTH.copy()
    truth[synth.X0], truth[synth.Y0] = 0.5 * (g.nx - 1), 0.5 * (g.ny - 1)
    maps = G.eval_maps(g, torch.from_numpy(truth[None])).cpu().numpy()[0]
    wv, ws = synth.weights(shape, 5.0)
    return G.Obs.from_numpy((maps[1] + rng.normal(0, 5, shape)).astype(np.float32),
                            (maps[2] + rng.normal(0, 7.07, shape)).astype(np.float32), wv, ws,
                            synth.dead_fibre_mask(rng, shape))


def _noalloc(G, g, dp, obs, n):
    out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    res = torch.full((n, 2, g.ny, g.nx), -1.0, dtype=torch.float32, device="cuda")
    cg = G.cgeom(g)
    st = G.lib().gbk_chi2_noalloc(ctypes.byref(cg), n, ctypes.c_void_p(dp.data_ptr()), ctypes.byref(obs.c()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(res.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, G.lib().gbk_last_error().decode()
    torch.cuda.synchronize()
    return out.cpu().numpy(), res.cpu().numpy()


# Both paths run the same deterministic kernels on the same inputs, so the
# results are identical bit for bit.  The calls go from a larger layout
# (a wider PSF, so another convolution kernel and longer rows, more models)
# to the smaller one and back, so the shared scratch holds another layout's
# leftovers at every call: nothing may depend on it starting at zero.
def test_noalloc_matches_workspace_path_on_two_calls(G):
    big = synth.SINGLE_GEOM.with_(nx=40, ny=40, psf_fwhm=4.0, lsf_fwhm=40.0)
    cases = [(big, 10, 11), (synth.SINGLE_GEOM, 8, 12), (synth.SINGLE_GEOM, 8, 13), (big, 6, 14)]
    for call, (g, n, seed) in enumerate(cases):
        obs = _obs(G, g, seed)
        rng = np.random.default_rng(seed)
        truth = synth.SINGLE_TRUTH.copy()
        truth[synth.X0], truth[synth.Y0] = 0.5 * (g.nx - 1), 0.5 * (g.ny - 1)
        ps = np.array([synth.perturb(rng, truth) for _ in range(n)])
        dp = torch.from_numpy(ps).cuda()
        ref, ref_r = G.chi2(g, dp, obs, flags=G.PATH_STAGED, want_resid=True)
        out, res = _noalloc(G, g, dp, obs, n)
        np.testing.assert_array_equal(out, ref.cpu().numpy(), err_msg="call %d" % call)
        np.testing.assert_array_equal(res, ref_r.cpu().numpy(), err_msg="call %d" % call)


def test_noalloc_rejects_batches_beyond_its_scratch(G):
    g = synth.SINGLE_GEOM
    n = 200  # about 150 MB of staged scratch at 32 x 32 x 64
    assert G.gbk_workspace_bytes(g, n, G.PATH_STAGED) > (32 << 20)
    obs = _obs(G, g, 2)
    dp = torch.from_numpy(np.array([synth.SINGLE_TRUTH] * n)).cuda()
    out = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GbkError) as ei:
        G.gbk_chi2_noalloc(g, dp, obs, out)
    assert ei.value.status == G.GBK_EWORKSPACE
    torch.cuda.synchronize()
    assert torch.all(out == -1.0)  # nothing ran
