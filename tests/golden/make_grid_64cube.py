"""Writes grid_64cube.json: the FP64 oracle's nested-grid search (Sec. 2.3.3)
on the 64 x 64 x 64 cube with 10^5 nodes per level over (PA, i, V_max, r_t,
sigma0) and three levels -- the expected argmin index of every level for the
GPU test in tests/test_grid.py.

Only the oracle computes here (oracle.fit.grid_search, with the convolution
done as three 1-D passes, the same linear map as the direct 3-D sum); the
inputs are the seeded ones the test draws (truth from seed 3, observed maps
from the oracle at the truth plus N(0, 5) / N(0, 5 sqrt 2) noise of seed 31).

Run:  python tests/golden/make_grid_64cube.py      (about 15 min on 8 cores)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))                   # tests/ (cases)
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))  # repository root

import oracle  # noqa: E402
from oracle import fit  # noqa: E402
from cases import make_obs, ogeom  # noqa: E402
from grid64 import AXES, GEOM, LEVELS, NODES_PER_AXIS, box, truth  # noqa: E402

OUT = os.path.join(HERE, "grid_64cube.json")


def main():
    p_true = truth()
    obs = make_obs(GEOM, p_true, seed=31, noise_v=5.0, dead=0.0)
    lo, hi = box(p_true)
    nodes = [1] * 10
    for k in AXES:
        nodes[k] = NODES_PER_AXIS
    t = time.time()
    with oracle.separable_convolution():
        bp, bi, bc, allc = fit.grid_search(ogeom(GEOM), obs, lo, hi, nodes, p_true, levels=LEVELS)
    levels = []
    for lev in range(LEVELS):
        c = np.where(np.isnan(allc[lev]), np.inf, allc[lev])
        order = np.argsort(c, kind="stable")
        levels.append({"best_index": int(bi[lev]), "best_chi2": float(bc[lev]),
                       "second_index": int(order[1]), "second_chi2": float(c[order[1]]),
                       "n_nodes": int(c.size)})
    doc = {"what": "oracle nested grids, 64x64x64 cube, 10^5 nodes per level over (PA, i, Vmax, r_t, sigma0), "
                   "3 levels; written by tests/golden/make_grid_64cube.py from oracle/ only",
           "paper": "Sec. 2.3.3 (nested grids)",
           "truth": [float(v) for v in p_true], "lo": [float(v) for v in lo], "hi": [float(v) for v in hi],
           "best_params": [float(v) for v in bp], "levels": levels,
           "oracle_seconds": round(time.time() - t, 1)}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print(json.dumps(doc["levels"]), doc["oracle_seconds"], "s")


if __name__ == "__main__":
    main()
