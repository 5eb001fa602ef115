"""Failure detection without a GPU fault: a bounded device wait on a barrier
that nothing completes runs out, is reported through the device status word
(gbk_device_status, bit 2), and leaves the context usable."""
import numpy as np
import pytest
import torch

import oracle
from cases import ogeom, check_maps
from paper_1510_01815_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    from paper_1510_01815_gb300 import build, gbk
    build.build()
    assert torch.cuda.is_available()
    return gbk


def _maps_still_match(G):
    g, p = synth.SINGLE_GEOM, synth.SINGLE_TRUTH
    ref = oracle.evaluate_batch(ogeom(g), p[None])
    maps = G.eval_maps(g, torch.from_numpy(p[None])).cpu().numpy()
    check_maps(maps, ref, p[None], "after a timed-out wait")


def test_a_wait_nothing_completes_runs_out_and_is_reported(G):
    G.gbk_device_status()  # clear
    ns_out = G.gbk_wait_selfcheck(256, complete=False)
    assert G.gbk_device_status() == 4
    assert G.gbk_device_status() == 0  # read and cleared
    ns_done = G.gbk_wait_selfcheck(256, complete=True)
    assert G.gbk_device_status() == 0
    assert ns_out > ns_done >= 0
    _maps_still_match(G)
    assert G.gbk_device_status() == 0


def test_the_number_of_tries_bounds_the_wait(G):
    short = G.gbk_wait_selfcheck(16, complete=False)
    long_ = G.gbk_wait_selfcheck(1024, complete=False)
    assert G.gbk_device_status() == 4
    assert long_ > short
    assert long_ < 5e9  # well inside a second or so per thousand tries
