"""Nested grids (Sec. 2.3.3): the GPU's gbk_grid against the oracle's search
(argmin index per level) on the case the oracle's pins fix (tests/fit_pins.py)."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import fit
from cases import ogeom, make_obs
from fit_pins import (GRID_GEOM, GRID_HI, GRID_LO, GRID_NODES, GRID_TRUTH, GRID_TRUTH_INDEX,
                      grid_noiseless_obs)

# the case with the truth on a node, shared with the oracle's pins (fit_pins)
GEOM, TRUTH, NODES, LO, HI = GRID_GEOM, GRID_TRUTH, GRID_NODES, GRID_LO, GRID_HI
TRUTH_INDEX = GRID_TRUTH_INDEX
noiseless_obs = grid_noiseless_obs


@pytest.mark.gpu
@pytest.mark.parametrize("noise,chunk", [(0.0, 128), (5.0, 100), (5.0, 4096)])
def test_gpu_grid_argmin_matches_oracle(noise, chunk):
    import torch
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    if noise == 0.0:
        obs = noiseless_obs()
    else:
        obs = make_obs(GEOM, TRUTH, seed=17, noise_v=noise, dead=0.02)
    lo, hi = LO.copy(), HI.copy()
    lo[2], hi[2] = 35.0, 83.0  # truth off the nodes for the noisy cases
    if noise == 0.0:
        lo, hi = LO, HI
    levels = 3
    bp_o, bi_o, bc_o, allc = fit.grid_search(ogeom(GEOM), obs, lo, hi, NODES, TRUTH, levels=levels)
    dobs = gbk.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    bp, bi, bc = gbk.gbk_grid(GEOM, dobs, lo, hi, NODES, TRUTH, levels=levels, chunk=chunk)
    for lev in range(levels):
        c = np.sort(allc[lev])
        gap = c[1] - c[0]
        # a tie within the GPU's chi2 error (FP32 maps) cannot be decided
        if gap > 1e-3 * max(c[0], 1e-3):
            assert bi[lev] == bi_o[lev], (lev, bi, bi_o)
            assert abs(bc[lev] - bc_o[lev]) <= 1e-3 * max(bc_o[lev], 1e-3) + 1e-6, (bc, bc_o)
        else:
            break  # later levels depend on the undecided tie
    if noise == 0.0:
        assert bi[0] == TRUTH_INDEX


# Full-size nested grid (10^5 nodes per level over PA, i, V_max, r_t, sigma0;
# 3 levels) on a 64 x 64 x 64 cube (tests/grid64.py).  The expected argmin
# of every level is the FP64 oracle's, written by
# tests/golden/make_grid_64cube.py into tests/golden/grid_64cube.json.  Tie
# rule: the GPU's chi2 of a node differs from the oracle's by at most the
# bound its map deviations imply (cases.chi2_bound); a level is decided when
# the oracle's gap between its best and second-best node exceeds the sum of
# the two nodes' bounds, and then the GPU's index must equal the oracle's.
# A level that is not decided is reported as a tie within tolerance, and the
# levels after it (whose boxes depend on it) are not compared.
GOLDEN64 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid_64cube.json")


@pytest.mark.gpu
def test_gpu_grid_full_size_argmin_matches_oracle_golden():
    import torch
    import grid64
    from cases import chi2_bound
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    with open(GOLDEN64) as f:
        gold = json.load(f)
    truth = grid64.truth()
    np.testing.assert_array_equal(truth, np.array(gold["truth"]))  # same seeded case
    obs = make_obs(grid64.GEOM, truth, seed=31, noise_v=5.0, dead=0.0)
    lo, hi = grid64.box(truth)
    nodes = [1] * 10
    for k in grid64.AXES:
        nodes[k] = grid64.NODES_PER_AXIS
    dobs = gbk.Obs.from_numpy(obs.v, obs.s, obs.w_v, obs.w_s, obs.mask)
    bp, bi, bc = gbk.gbk_grid(grid64.GEOM, dobs, lo, hi, nodes, truth, levels=grid64.LEVELS, chunk=16384)
    og = ogeom(grid64.GEOM)
    clo, chi = lo.copy(), hi.copy()
    decided = 0
    for lev, L in enumerate(gold["levels"]):
        assert L["n_nodes"] == grid64.NODES_PER_AXIS ** len(grid64.AXES)
        steps = {k: (chi[k] - clo[k]) / (grid64.NODES_PER_AXIS - 1) for k in grid64.AXES}
        pair = np.array([grid64.node_params(L["best_index"], clo, steps, truth),
                         grid64.node_params(L["second_index"], clo, steps, truth)])
        gm = gbk.eval_maps(grid64.GEOM, torch.from_numpy(pair)).cpu().numpy()
        bounds = []
        for j, key in ((0, "best_chi2"), (1, "second_chi2")):
            ref_maps = oracle.evaluate(og, pair[j])
            bounds.append(chi2_bound(ref_maps, gm[j], obs, L[key]))
        gap = L["second_chi2"] - L["best_chi2"]
        if not gap > bounds[0] + bounds[1]:
            print("level %d: tie within tolerance (gap %.3g, bounds %.3g + %.3g)" % (lev, gap, *bounds))
            break
        assert int(bi[lev]) == L["best_index"], (lev, int(bi[lev]), L["best_index"], gap, bounds)
        assert abs(bc[lev] - L["best_chi2"]) <= bounds[0], (lev, bc[lev], L["best_chi2"], bounds[0])
        decided += 1
        best = pair[0]
        for k in grid64.AXES:
            clo[k] = max(lo[k], best[k] - steps[k])
            chi[k] = min(hi[k], best[k] + steps[k])
    assert decided >= 1, "the first level of the golden case must be decidable"
    if decided == grid64.LEVELS:
        np.testing.assert_allclose(bp, np.array(gold["best_params"]), rtol=1e-12, atol=1e-12)
    # the final node recovers what the data fix: PA, and V_max sin i (V_max and
    # i alone slide along the degeneracy valley of Sec. 6.1, which a grid
    # refined around its first level's choice cannot leave)
    vs, vs_t = bp[5] * np.sin(np.radians(bp[3])), truth[5] * np.sin(np.radians(truth[3]))
    assert abs(vs - vs_t) < 0.03 * vs_t, (bp, truth)
    assert abs(((bp[2] - truth[2] + 180) % 360) - 180) < 3.0, (bp, truth)
