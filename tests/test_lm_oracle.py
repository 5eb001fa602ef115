"""The oracle's Levenberg-Marquardt (Sec. 2.3.1) against what the paper
reports for zero-noise mock data (Sec. 4.1, Tables 3-4): from perturbed
starts, recovered V_t within 2 km/s and PA within 1 degree; and against the
exact minimum of noiseless data (chi2 -> 0)."""
import numpy as np

import oracle
from oracle import fit
from cases import ogeom
from lm_cases import FREE, bounds, galaxy, starts
from paper_1510_01815_gb300 import synth


def test_oracle_lm_recovers_noiseless_parameters():
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    for p0 in starts(p, 2, seed=3):
        q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, FREE, max_iter=100)
        assert st in (fit.FTOL, fit.XTOL), (st, it)
        assert abs(q[synth.VMAX] - p[synth.VMAX]) < 2.0, q
        assert abs(q[synth.PA] - p[synth.PA]) < 1.0, q
        assert c < 1e-6, c


def test_oracle_lm_solves_a_linear_problem_in_one_step():
    """With only V_sys free the residual is linear in the parameter (a shift
    of every velocity), so the undamped Gauss-Newton step is exact; with the
    default damping lambda0 = 1e-3 the first step lands within 0.1 percent."""
    g, p, obs = galaxy(noise_v=0.0)
    lo, hi = bounds(p)
    p0 = p.copy()
    p0[synth.VSYS] = 25.0
    q, c, it, st = fit.fit_lm(ogeom(g), obs, p0, lo, hi, [synth.VSYS], max_iter=1, fd_step=0.1)
    assert abs(q[synth.VSYS]) < 25.0 * 2e-3, q[synth.VSYS]
