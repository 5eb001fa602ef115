"""The mock-dataset study (Sec. 3.1, results in Sec. 4.1) at reduced size:
galaxies over the mock parameter space fitted by the batched LM.  On the
clean dataset nearly every galaxy is recovered within the paper's
thresholds; on noisy data the standardised residuals (fit - truth over the
1-sigma error from the Fisher matrix of the analytic Jacobian) fall within
1 and 2 sigma at about the Gaussian rates (68 and 95 per cent)."""
import numpy as np
import pytest
import torch

import bench
from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def test_clean_mock_recovery(G):
    truth, q, it, st, err, dt = bench.mock_study(G, torch, 96, 0.0, 31, "cuda")
    assert err is None
    d = bench.mock_residuals(truth, q)
    # thin discs near edge-on and the V_t - i degeneracy near face-on are
    # the paper's few failures; the rest is recovered
    for k, t in bench.MOCK_THRESHOLDS.items():
        assert np.mean(d[:, k] < t) >= 0.9, (synth.PARAM_NAMES[k], np.mean(d[:, k] < t))
    assert np.median(d[:, synth.VMAX]) < 0.5 and np.median(d[:, synth.PA]) < 0.05
    assert np.mean(np.isin(st, [1, 2])) >= 0.95


def test_noisy_mock_standardised_residuals(G):
    truth, q, it, st, err, dt = bench.mock_study(G, torch, 96, 5.0, 36, "cuda")
    free = list(bench.FIT_FREE)
    d = bench.mock_residuals(truth, q)[:, free]
    z = d / err
    ok = np.isfinite(z).all(axis=1)
    assert np.mean(ok) >= 0.95
    w1 = np.mean(z[ok] < 1.0)
    w2 = np.mean(z[ok] < 2.0)
    # all parameters pooled (about 700 values): Gaussian 0.683 and 0.954
    assert 0.58 < w1 < 0.78, (w1, w2)
    assert 0.88 < w2 < 0.99, (w1, w2)
