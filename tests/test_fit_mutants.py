"""Plant plausible mistakes in copies of the oracle's optimisers
(oracle/fit.py) and check that the pins catch every one (fastest pins first;
a mutant counts as caught at the first pin that fails).  A copy is loaded as
a module of the oracle package, so its relative imports resolve."""
import importlib.util
import os

import pytest

from oracle import fit
from fit_pins import ALL_FIT_PINS

SRC = fit.__file__

MUTANTS = [
    ("lm_step_uphill", "y = np.linalg.solve(L, -JTr)", "y = np.linalg.solve(L, JTr)"),
    ("lm_accepts_rises", "if np.isfinite(ct) and ct <= cc and dn > 0:", "if np.isfinite(ct) and ct >= cc and dn > 0:"),
    ("lm_jacobian_sign", "J = np.stack([(r[1 + j].ravel() - r0) / hs[j] for j in range(nf)], axis=1)",
     "J = np.stack([(r0 - r[1 + j].ravel()) / hs[j] for j in range(nf)], axis=1)"),
    ("lm_central_step_not_doubled", "hs.append(2 * h)", "hs.append(h)"),
    ("lm_central_minus_side_forward", "q[k] = p[k] - steps[k]", "q[k] = p[k] + steps[k]"),
    ("lm_trial_not_clipped", "pt[k] = min(max(p[k] + d[j], lo[k]), hi[k])", "pt[k] = p[k] + d[j]"),
    ("lm_damping_grows_on_success", "lam = max(lam * max(0.1, 1.0 - (2.0 * rho - 1.0) ** 3), 1e-12)",
     "lam = lam * 10.0"),
    ("lm_predicted_decrease_sign", "pred = -(2.0 * (s @ JTr) + s @ JTJ @ s)", "pred = 2.0 * (s @ JTr) + s @ JTJ @ s"),
    ("lm_predicted_decrease_drops_curvature", "pred = -(2.0 * (s @ JTr) + s @ JTJ @ s)", "pred = -(2.0 * (s @ JTr))"),
    ("lm_rejection_factor_fixed", "            nu *= 2.0\n", "            nu *= 1.0\n"),
    ("lm_rejection_tenfold", "            lam *= nu\n", "            lam *= 10.0\n"),
    ("grid_nan_not_worst", "key = np.where(np.isnan(c), np.inf, c)", "key = c"),
    ("grid_column_major", "mesh = np.meshgrid(*grids, indexing=\"ij\")", "mesh = np.meshgrid(*grids, indexing=\"xy\")"),
    ("grid_steps_off_by_one", "steps = {k: (chi[k] - clo[k]) / (nodes[k] - 1) for k in axes}",
     "steps = {k: (chi[k] - clo[k]) / nodes[k] for k in axes}"),
    ("grid_box_not_shrunk_below", "clo[k] = max(lo[k], bp[k] - steps[k])", "clo[k] = lo[k]"),
    ("grid_box_two_steps", "chi[k] = min(hi[k], bp[k] + steps[k])", "chi[k] = min(hi[k], bp[k] + 2 * steps[k])"),
    ("splitmix_increment", "self.s = (self.s + 0x9E3779B97F4A7C15) & self.M", "self.s = (self.s + 0x9E3779B97F4A7C13) & self.M"),
    ("ns_shrinks_twice_as_fast", "logx -= 1.0 / N", "logx -= 2.0 / N"),
    ("ns_takes_worse_points", "if not lp[j] > logl[w]:", "if not lp[j] < logl[w]:"),
    ("ns_final_live_points_unweighted", "lw = logx - np.log(N) + logl[i]", "lw = logx + logl[i]"),
    ("ns_posterior_weights_unnormalised", "wgt = np.exp(np.array(dead_lw) - logz)", "wgt = np.exp(np.array(dead_lw))"),
    ("ns_nan_likelihood_outside_domain", "return np.where(np.isfinite(c), -0.5 * c, -np.inf)", "return -0.5 * c"),
    ("ns_trace_records_the_best_not_the_worst", "w = int(np.argmin(logl))", "w = int(np.argmax(logl))"),
]


def _load(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(str(tmp_path), "fit_%s.py" % name)
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle.fit_" + name, path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(name, old, new, tmp_path):
    mod = _load(name, old, new, tmp_path)
    for pin in ALL_FIT_PINS:
        try:
            pin(mod)
        except (AssertionError, ValueError, IndexError, FloatingPointError, OverflowError):
            return
    pytest.fail("no pin catches the mutant %s" % name)
