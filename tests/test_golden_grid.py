"""The stored full-size nested-grid golden (tests/golden/grid_64cube.json,
written from the oracle by tests/golden/make_grid_64cube.py with the
convolution as three 1-D passes) checked against the oracle's definition:
the chi2 of each level's best and second-best node, recomputed with the
direct 3-D convolution, equals the stored value, and each level's box is
the previous level's best node +- one step, clipped to the prior box
(Sec. 2.3.3)."""
import json
import os

import numpy as np

import oracle
import grid64
from cases import make_obs, ogeom

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "grid_64cube.json")


def test_golden_grid_nodes_match_direct_oracle():
    with open(GOLDEN) as f:
        gold = json.load(f)
    truth = grid64.truth()
    np.testing.assert_array_equal(truth, np.array(gold["truth"]))
    obs = make_obs(grid64.GEOM, truth, seed=31, noise_v=5.0, dead=0.0)
    lo, hi = grid64.box(truth)
    np.testing.assert_array_equal(lo, gold["lo"])
    np.testing.assert_array_equal(hi, gold["hi"])
    clo, chi = lo.copy(), hi.copy()
    og = ogeom(grid64.GEOM)
    for L in gold["levels"]:
        steps = {k: (chi[k] - clo[k]) / (grid64.NODES_PER_AXIS - 1) for k in grid64.AXES}
        pair = np.array([grid64.node_params(L["best_index"], clo, steps, truth),
                         grid64.node_params(L["second_index"], clo, steps, truth)])
        c = oracle.chi2_batch(og, pair, obs)  # direct 3-D convolution
        np.testing.assert_allclose(c, [L["best_chi2"], L["second_chi2"]], rtol=1e-9)
        assert L["best_chi2"] <= L["second_chi2"]
        for k in grid64.AXES:
            clo[k] = max(lo[k], pair[0][k] - steps[k])
            chi[k] = min(hi[k], pair[0][k] + steps[k])
    np.testing.assert_allclose(np.array(gold["best_params"]),
                               grid64.node_params(gold["levels"][-1]["best_index"],
                                                  *_last_box(gold, lo, hi, truth)), rtol=1e-12)


def _last_box(gold, lo, hi, truth):
    clo, chi = lo.copy(), hi.copy()
    for L in gold["levels"][:-1]:
        steps = {k: (chi[k] - clo[k]) / (grid64.NODES_PER_AXIS - 1) for k in grid64.AXES}
        b = grid64.node_params(L["best_index"], clo, steps, truth)
        for k in grid64.AXES:
            clo[k] = max(lo[k], b[k] - steps[k])
            chi[k] = min(hi[k], b[k] + steps[k])
    steps = {k: (chi[k] - clo[k]) / (grid64.NODES_PER_AXIS - 1) for k in grid64.AXES}
    return clo, steps, truth
