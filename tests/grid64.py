"""The full-size nested-grid case (Sec. 2.3.3): a 64 x 64 x 64 cube at
20 km/s with the PSF and LSF of the single-galaxy workload, 10 nodes on each
of PA, i, V_max, r_t and sigma0 (10^5 nodes per level), three levels, the
other parameters fixed at the truth.  Shared by the golden-writing script
(tests/golden/make_grid_64cube.py) and the GPU test."""
import numpy as np

from paper_1510_01815_gb300.synth import Geometry, params as P

GEOM = Geometry(64, 64, 64, 20.0, 0.0, 2.5, 30.0)
AXES = (2, 3, 5, 6, 7)          # PA, i, Vmax, r_t, sigma0 (row-major order, PA slowest)
NODES_PER_AXIS = 10
LEVELS = 3
RANGES = {2: (0.0, 360.0), 3: (20.0, 80.0), 5: (50.0, 300.0), 6: (1.0, 8.0), 7: (10.0, 80.0)}


def truth():
    """Drawn once from the Fabry-Perot workload's ranges (seed 3)."""
    rng = np.random.default_rng(3)
    return P(31.5, 31.5, rng.uniform(0, 360), rng.uniform(20, 80), 0.0, rng.uniform(50, 300),
             rng.uniform(1, 8), rng.uniform(10, 80), 1.0, 8.0)


def box(p_true):
    lo, hi = p_true.copy(), p_true.copy()
    for k, (a, b) in RANGES.items():
        lo[k], hi[k] = a, b
    return lo, hi


def node_params(i, box_lo, steps, fixed):
    """Parameters of node i (row-major over AXES) of a level whose grid starts
    at box_lo with the given per-axis steps."""
    p = np.array(fixed, dtype=np.float64)
    idx = np.unravel_index(int(i), [NODES_PER_AXIS] * len(AXES))
    for a, k in enumerate(AXES):
        p[k] = box_lo[k] + idx[a] * steps[k]
    return p
