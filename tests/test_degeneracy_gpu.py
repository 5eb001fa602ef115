"""The V_t - i degeneracy (Sec. 6.1): reduced chi-squared maps over the
(inclination, circular velocity) plane of mock galaxies with V_t = 200 km/s
at i = 20, 40, 60 and 70 degrees and 5 km/s noise, every node one model of a
single gbk_chi2 launch.  The map agrees with the FP64 oracle node by node,
and it shows the degeneracy the paper describes: below 40 degrees the
confidence region stretches along V_t sin i = const, above it shrinks to a
small ellipse."""
import numpy as np
import pytest
import torch

import oracle
from cases import chi2_bound, ogeom
from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu

G_ = synth.SINGLE_GEOM
INC = np.arange(5.0, 85.0 + 1e-9, 0.25)
VT = np.arange(50.0, 600.0 + 1e-9, 1.0)
# chi-squared increments of the 1 and 3 sigma regions of two parameters
D1, D3 = 2.30, 11.83


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def _truth(inc):
    p = synth.SINGLE_TRUTH.copy()
    p[synth.INCL], p[synth.VMAX] = inc, 200.0
    return p


def _obs(inc):
    m = oracle.evaluate(ogeom(G_), _truth(inc))
    rng = np.random.default_rng(100 + int(inc))
    wv, ws = synth.weights((G_.ny, G_.nx), 5.0)
    v = (m[1] + rng.normal(0.0, 5.0, m[1].shape)).astype(np.float32)
    s = (m[2] + rng.normal(0.0, 5.0 * np.sqrt(2.0), m[2].shape)).astype(np.float32)
    return oracle.Obs(v, s, wv, ws, np.ones((G_.ny, G_.nx), np.uint8))


def _grid(p):
    ii, vv = np.meshgrid(INC, VT, indexing="ij")
    grid = np.repeat(p[None], ii.size, 0)
    grid[:, synth.INCL], grid[:, synth.VMAX] = ii.ravel(), vv.ravel()
    return grid, ii, vv


def _map(G, inc):
    obs = _obs(inc)
    grid, ii, vv = _grid(_truth(inc))
    d = G.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    c = G.chi2(G_, torch.from_numpy(grid), d).cpu().numpy().reshape(ii.shape)
    return obs, grid, ii, vv, c


@pytest.mark.parametrize("inc", [20.0, 60.0])
def test_chi2_map_matches_oracle(G, inc):
    """Sampled nodes of the map against the oracle, within the bound that
    the measured map deviations imply."""
    obs, grid, ii, vv, c = _map(G, inc)
    rng = np.random.default_rng(7)
    pick = rng.choice(grid.shape[0], size=48, replace=False)
    pick[0] = int(np.argmin(c))  # and the best node
    gm = G.eval_maps(G_, torch.from_numpy(grid[pick])).cpu().numpy()
    for n, k in enumerate(pick):
        ref_maps = oracle.evaluate(ogeom(G_), grid[k])
        ref_c = oracle.chi2_maps(ref_maps, obs)
        b = chi2_bound(ref_maps, gm[n], obs, ref_c)
        assert abs(c.ravel()[k] - ref_c) <= b, (k, c.ravel()[k], ref_c, b)


def test_degeneracy_shape(G):
    ext = {}
    for inc in (20.0, 40.0, 60.0, 70.0):
        _, _, ii, vv, c = _map(G, inc)
        dof = 2 * G_.nx * G_.ny - 2
        assert 0.9 < c.min() / dof < 1.1, (inc, c.min() / dof)  # noise at the expected level
        d = c - c.min()
        r1, r3 = d <= D1, d <= D3
        # the truth lies inside the 3 sigma region
        assert d[np.argmin(np.abs(INC - inc)), np.argmin(np.abs(VT - 200.0))] <= D3, inc
        vs = vv[r3] * np.sin(np.radians(ii[r3]))
        ext[inc] = (np.ptp(vv[r1]), np.ptp(vv[r3]), np.ptp(ii[r3]), np.ptp(vs) / np.mean(vs))
    # V_t is poorly constrained at 20 degrees and well constrained at 60-70
    assert ext[20.0][1] > 100.0, ext
    assert ext[70.0][1] < 20.0 and ext[60.0][1] < 25.0, ext
    assert ext[20.0][1] > 5.0 * ext[60.0][1], ext
    # along the valley the product V_t sin i is what the data fix
    assert ext[20.0][3] < 0.05, ext
    # the region shrinks monotonically with inclination
    assert ext[20.0][1] > ext[40.0][1] > ext[70.0][1], ext
