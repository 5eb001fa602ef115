"""The two-stage kernels inside a caller's CUDA graph.

A call over several chunks of models forks its PSF stages onto an auxiliary
stream and joins them back before it returns; under stream capture that
fork and join become graph dependencies.  A captured call, replayed, must
give the eager call's results bit for bit, and a replay must see new inputs
written in place (the graph holds pointers, not values)."""
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


def _obs(G, g, p, seed):
    maps = G.eval_maps(g, torch.from_numpy(p[None]))
    rng = np.random.default_rng(seed)
    m = maps[0].cpu().numpy()
    shape = (g.ny, g.nx)
    v = (m[1] + rng.normal(0, 5.0, shape)).astype(np.float32)
    s = (m[2] + rng.normal(0, 5.0 * np.sqrt(2.0), shape)).astype(np.float32)
    wv, ws = synth.weights(shape, 5.0)
    return G.Obs.from_numpy(v, s, wv, ws, np.ones(shape, np.uint8))


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        fn(side)  # warm-up outside the capture: kernel attributes and the auxiliary stream
        side.synchronize()
        with torch.cuda.graph(graph, stream=side):
            fn(side)
    torch.cuda.current_stream().wait_stream(side)
    return graph


def test_split_evaluator_in_a_captured_graph(G):
    """400 Fabry-Perot models (five chunks, both plane buffers, the PSF
    stages on the auxiliary stream): the replayed graph's chi2 equals the
    eager call's, before and after the parameters are rewritten in place."""
    g = synth.FP_GEOM
    rng = np.random.default_rng(3)
    p = synth.draw_fp_params(rng, 400)
    obs = _obs(G, g, p[0], 4)
    d_p = torch.from_numpy(p).cuda()
    ws = torch.empty(G.gbk_workspace_bytes(g, 400, G.PATH_SPLIT), dtype=torch.uint8, device="cuda")
    eager = torch.empty(400, dtype=torch.float64, device="cuda")
    G.gbk_chi2(g, d_p, obs, eager, None, G.PATH_SPLIT, ws)
    torch.cuda.synchronize()
    out = torch.empty_like(eager)
    graph = _capture(lambda st: G.gbk_chi2(g, d_p, obs, out, None, G.PATH_SPLIT, ws, st))
    out.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    p2 = synth.draw_fp_params(rng, 400)
    d_p.copy_(torch.from_numpy(p2))
    graph.replay()
    G.gbk_chi2(g, d_p, obs, eager, None, G.PATH_SPLIT, ws)
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


def test_split_jacobian_in_a_captured_graph(G):
    """2048 C1 models (seven chunks): J^T J, J^T r and chi2 from a replayed
    graph equal the eager call's."""
    g = synth.SINGLE_GEOM
    n = 2048
    rng = np.random.default_rng(5)
    truth = synth.SINGLE_TRUTH
    p = np.array([synth.perturb(rng, truth, synth.FREE_DEFAULT, 0.2) for _ in range(n)])
    obs = _obs(G, g, truth, 6)
    d_p = torch.from_numpy(p).cuda()
    ws = torch.empty(G.gbk_jacobian_workspace_bytes(g, n), dtype=torch.uint8, device="cuda")
    outs = [[torch.empty((n, 8, 8), dtype=torch.float64, device="cuda"),
             torch.empty((n, 8), dtype=torch.float64, device="cuda"),
             torch.empty(n, dtype=torch.float64, device="cuda")] for _ in range(2)]
    G.gbk_jacobian_ws(g, d_p, obs, jtj=outs[0][0], jtv=outs[0][1], chi2=outs[0][2], workspace=ws)
    torch.cuda.synchronize()
    graph = _capture(lambda st: G.gbk_jacobian_ws(g, d_p, obs, jtj=outs[1][0], jtv=outs[1][1], chi2=outs[1][2],
                                                  workspace=ws, stream=st))
    for t in outs[1]:
        t.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs[0], outs[1]):
        assert torch.equal(a, b)
