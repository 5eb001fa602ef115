"""The C ABI: the library builds, loads and exports every symbol include/gbk.h
declares; host-side validation rejects bad arguments before any launch.
These tests make no compute calls and need no GPU."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1510_01815_gb300 import build as gbuild
from paper_1510_01815_gb300.synth import SINGLE_GEOM, FP_GEOM, GRID_GEOM

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbk.h")


@pytest.fixture(scope="module")
def gbk():
    gbuild.build()
    from paper_1510_01815_gb300 import gbk as G
    G.lib()
    return G


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GBK_API\s+[\w\s\*]*?\b(gbk_\w+)\s*\(", text)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("gbk_eval_cubes", "gbk_chi2", "gbk_workspace_bytes", "gbk_last_error"):
        assert s in syms


def test_every_declared_symbol_is_exported(gbk):
    out = subprocess.run(["nm", "-D", "--defined-only", gbk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(gbk_\w+)", out))
    for s in declared_symbols():
        assert s in exported, s
        assert hasattr(gbk.lib(), s)
    assert set(gbk.exported_symbols()) <= exported


def test_no_stray_exports(gbk):
    out = subprocess.run(["nm", "-D", "--defined-only", gbk.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)", out))
    extra = {s for s in exported if s.startswith("gbk_")} - set(declared_symbols())
    assert not extra, extra


def test_version(gbk):
    assert "sm_103a" in gbk.gbk_version()


def test_workspace_sizes(gbk):
    # fused path needs none; the staged path holds the extended cube, the data
    # cube and the chi2 partials
    assert gbk.gbk_workspace_bytes(SINGLE_GEOM, 10, gbk.PATH_FUSED) == 0
    assert gbk.gbk_workspace_bytes(SINGLE_GEOM, 10, gbk.PATH_AUTO) == gbk.gbk_workspace_bytes(SINGLE_GEOM, 10,
                                                                                               gbk.PATH_SPLIT) > 0
    n = 7
    ws = gbk.gbk_workspace_bytes(SINGLE_GEOM, n, gbk.PATH_STAGED)
    # 32x32x64, R = 5 (PSF FWHM 2.5), Rz = 3 (LSF 30 km/s at 20 km/s)
    ext = 70 * 42 * 44 * 4 * n      # row pitch 42 -> 44
    data = 64 * 32 * 32 * 4 * n
    part = 4 * 8 * n
    al = lambda b: (b + 255) // 256 * 256
    assert ws == al(ext) + al(data) + al(part)
    assert gbk.gbk_workspace_bytes(GRID_GEOM.with_(upsample=2), 1, gbk.PATH_AUTO) > 0
    # split path: per-model constants (60 B), the tables (taps and LSF edge
    # tables: 24 + 3 x 12 floats at Rz = 3), then for the models of a chunk
    # four x-filtered planes of ey x pad4(nx) floats (42 x 32), one chi2 part
    # per 64 x 32 tile and an arrival counter
    assert gbk.gbk_workspace_bytes(SINGLE_GEOM, n, gbk.PATH_SPLIT) == \
        al(60 * n) + al(4 * (24 + 3 * 12)) + al(4 * 42 * 32 * 4 * n) + al(8 * n) + al(4 * n)
    # the Fabry-Perot geometry: chunks of 48 MiB / (4 x 204 x 192 x 4 B) = 80
    # models, two plane buffers (a chunk's PSF stage beside the next chunk's
    # line stage)
    fp = gbk.gbk_workspace_bytes(FP_GEOM, 400, gbk.PATH_SPLIT)
    assert fp == al(60 * 400) + al(4 * (24 + 3 * 24)) + al(2 * 4 * 204 * 192 * 4 * 80) + al(8 * 18 * 80) + al(4 * 80)
    # the host-buffer call adds the device copies of the parameters, chi2 and
    # the five maps
    assert gbk.gbk_chi2_host_workspace_bytes(FP_GEOM, 400) == \
        al(8 * 10 * 400) + al(8 * 400) + al(4 * 4 * 192 * 192) + al(192 * 192) + fp


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(nz=-1), dict(dv=0.0), dict(dv=float("nan")), dict(psf_fwhm=-1.0),
    dict(lsf_mode=2), dict(upsample=0), dict(halo_sigmas=0.0), dict(psf_fwhm=1e4)])
def test_invalid_geometry_rejected(gbk, bad):
    g = SINGLE_GEOM.with_(**bad)
    with pytest.raises(gbk.GbkError) as ei:
        gbk.gbk_workspace_bytes(g, 1, gbk.PATH_STAGED)
    assert ei.value.status in (gbk.GBK_EINVAL, gbk.GBK_EUNSUPPORTED)
    cg = gbk.cgeom(g)
    st = gbk.lib().gbk_eval_cubes(ctypes.byref(cg), 1, None, None, None, None, 0, None)
    assert st in (gbk.GBK_EINVAL, gbk.GBK_EUNSUPPORTED)
    assert gbk.lib().gbk_last_error().decode()


def test_zero_models_is_a_noop(gbk):
    cg = gbk.cgeom(SINGLE_GEOM)
    assert gbk.lib().gbk_eval_cubes(ctypes.byref(cg), 0, None, None, None, None, 0, None) == 0
    assert gbk.lib().gbk_chi2(ctypes.byref(cg), 0, None, None, None, None, 0, None, 0, None) == 0


def test_null_and_host_pointers_rejected(gbk):
    cg = gbk.cgeom(SINGLE_GEOM)
    assert gbk.lib().gbk_eval_cubes(ctypes.byref(cg), 1, None, None, None, None, 0, None) == gbk.GBK_EINVAL
    host = (ctypes.c_double * 10)()
    st = gbk.lib().gbk_eval_cubes(ctypes.byref(cg), 1, ctypes.cast(host, ctypes.c_void_p), None, None,
                                  None, 0, None)
    assert st == gbk.GBK_EINVAL
    assert "params" in gbk.lib().gbk_last_error().decode()


def test_bad_flags_rejected(gbk):
    cg = gbk.cgeom(FP_GEOM)
    st = gbk.lib().gbk_chi2(ctypes.byref(cg), 1, None, None, None, None, 99, None, 0, None)
    assert st == gbk.GBK_EINVAL


def test_tuning_host_logic(gbk):
    """Heuristic default, forced tunings and their validation (no GPU)."""
    from paper_1510_01815_gb300.synth import Geometry
    g = FP_GEOM
    t = gbk.gbk_get_tuning(g)
    assert 1 <= t["cluster_ctas"] <= 16 and t["threads"] in (256, 384, 512)
    gbk.gbk_set_tuning(g, 8, 512, 1)
    assert gbk.gbk_get_tuning(g) == {"cluster_ctas": 8, "threads": 512, "persistent": 1}
    with pytest.raises(gbk.GbkError):
        gbk.gbk_set_tuning(g, 8, 512, 2)
    with pytest.raises(gbk.GbkError):
        gbk.gbk_set_tuning(g, 17, 512)
    with pytest.raises(gbk.GbkError):
        gbk.gbk_set_tuning(g, 8, 300)
    with pytest.raises(gbk.GbkError):      # one CTA cannot hold a 204-row band
        gbk.gbk_set_tuning(g, 1, 512)
    gbk.gbk_set_tuning(g, None)
    assert gbk.gbk_get_tuning(g) == t
    small = Geometry(3, 5, 7, 40.0, 0.0, 1.5, 50.0)
    assert gbk.gbk_get_tuning(small)["cluster_ctas"] >= 1
    with pytest.raises(gbk.GbkError):      # upsampled geometries use the staged path
        gbk.gbk_get_tuning(SINGLE_GEOM.with_(upsample=2))


def test_jacobian_and_lm_validation(gbk):
    import torch
    g = SINGLE_GEOM
    with pytest.raises(gbk.GbkError):
        gbk.gbk_fit_lm_workspace_bytes(g, 4, gbk.lm_opts(free=()))
    with pytest.raises(gbk.GbkError):
        gbk.gbk_fit_lm_workspace_bytes(g, 4, gbk.lm_opts(max_iter=0))
    with pytest.raises(gbk.GbkError):
        gbk.gbk_fit_lm_workspace_bytes(g, 4, gbk.lm_opts(jacobian=gbk.JAC_TANGENT, mode=gbk.LM_PLAIN))
    assert gbk.gbk_fit_lm_workspace_bytes(g, 4, gbk.lm_opts()) > 0
    # tangent mode needs no finite-difference batch
    assert (gbk.gbk_fit_lm_workspace_bytes(g, 64, gbk.lm_opts(jacobian=gbk.JAC_TANGENT))
            < gbk.gbk_fit_lm_workspace_bytes(g, 64, gbk.lm_opts()))
    cg = gbk.cgeom(g)
    st = gbk.lib().gbk_jacobian(ctypes.byref(cg), 1, None, None, 0, None, None, None, None, None, None)
    assert st == gbk.GBK_EINVAL
    # the seeded fit with a fallback needs the fit's workspace plus room for
    # the packed rows of every galaxy, and rejects what gbk_fit_lm rejects
    o = gbk.lm_opts()
    assert gbk.gbk_fit_lm_fallback_workspace_bytes(g, 64, o) > gbk.gbk_fit_lm_workspace_bytes(g, 64, o)
    with pytest.raises(gbk.GbkError):
        gbk.gbk_fit_lm_fallback_workspace_bytes(g, 4, gbk.lm_opts(free=()))
    st = gbk.lib().gbk_fit_lm_fallback(ctypes.byref(cg), 4, None, None, None, None, None, None, ctypes.byref(o),
                                       None, None, None, None, None, 0, None)
    assert st == gbk.GBK_EWORKSPACE
    assert gbk.lib().gbk_fit_lm_fallback(ctypes.byref(cg), 0, None, None, None, None, None, None, ctypes.byref(o),
                                         None, None, None, None, None, 0, None) == gbk.GBK_OK
    # the wait self-check validates its arguments before any launch
    assert gbk.lib().gbk_wait_selfcheck(0, 0, None, None) == gbk.GBK_EINVAL
    assert gbk.lib().gbk_wait_selfcheck((1 << 24) + 1, 0, None, None) == gbk.GBK_EINVAL
    assert gbk.lib().gbk_wait_selfcheck(16, 2, None, None) == gbk.GBK_EINVAL


def test_survey_host_logic(gbk):
    """Survey planning is host-only: sizes, validation and the rule that the
    workspace holds the geometry tables plus the LM state."""
    from paper_1510_01815_gb300 import synth
    import numpy as np
    gal = synth.draw_survey(np.random.default_rng(4), 16)
    geoms = [g for g, _ in gal]
    tables = gbk.gbk_survey_workspace_bytes(geoms)
    assert tables >= 16 * 64 and tables % 256 == 0
    lm = gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts())
    pix = sum(g.nx * g.ny for g in geoms)
    # FD batch of 1 + 8 models per galaxy, two residual maps each
    assert lm >= tables + 9 * 2 * pix * 4
    # the plain mode needs room for one galaxy at a time
    assert gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts(mode=gbk.LM_PLAIN)) < lm
    assert gbk.gbk_survey_workspace_bytes([], None) == 0
    # the cluster Jacobian needs no finite-difference batch
    cluster = gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts(jacobian=gbk.JAC_TANGENT, path=gbk.PATH_FUSED))
    assert tables < cluster < lm
    # the ragged split Jacobian (the default) adds its planes: 28 per
    # extended spaxel of the galaxies, up to an L2-sized chunk
    rag = gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts(jacobian=gbk.JAC_TANGENT))
    ext = sum((g.nx + 2 * 7) * (g.nx + 3) for g in geoms)
    assert rag > cluster and rag >= tables + 28 * 4 * ext
    assert gbk.gbk_survey_jacobian_workspace_bytes(geoms) > tables
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_jacobian_workspace_bytes(geoms, free=(synth.I0,))
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts(jacobian=gbk.JAC_TANGENT, path=gbk.PATH_STAGED))
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_workspace_bytes(geoms, gbk.lm_opts(jacobian=gbk.JAC_TANGENT, mode=gbk.LM_PLAIN))
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_workspace_bytes(geoms + [SINGLE_GEOM.with_(upsample=2)])
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_workspace_bytes(geoms + [SINGLE_GEOM.with_(nx=0)])
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_workspace_bytes([SINGLE_GEOM.with_(nx=2048, ny=2048)])
    cg = gbk.cgeoms(geoms)
    assert gbk.lib().gbk_survey_eval(cg, len(geoms), None, None, None, None, None, None, 0, None) == gbk.GBK_EINVAL


def test_survey_tuning_host_logic(gbk):
    """Survey launch shapes are planned on the host: one persistent launch by
    default, at the smallest cluster size that fits every galaxy; a forced
    shape must fit every galaxy; forgetting restores the default."""
    from paper_1510_01815_gb300 import synth
    import numpy as np
    geoms = [g for g, _ in synth.draw_survey(np.random.default_rng(4), 64)]
    t = gbk.gbk_survey_get_tuning(geoms)
    assert t["persistent"] == 1 and t["threads"] == 512 and 1 <= t["cluster_ctas"] <= 16
    cs = t["cluster_ctas"]
    small = [g for g in geoms if g.nx <= 40]
    assert gbk.gbk_survey_get_tuning(small)["cluster_ctas"] <= cs
    # one cluster size smaller than the default does not fit the largest galaxy
    # at two CTAs per SM, but may at one; anything at or above the default fits
    gbk.gbk_survey_set_tuning(geoms, 1, cs + 1, 256)
    assert gbk.gbk_survey_get_tuning(geoms) == {"cluster_ctas": cs + 1, "threads": 256, "persistent": 1}
    gbk.gbk_survey_set_tuning(geoms, 0)
    assert gbk.gbk_survey_get_tuning(geoms) == {"cluster_ctas": 0, "threads": 0, "persistent": 0}
    # the tuning belongs to this survey only
    assert gbk.gbk_survey_get_tuning(geoms[:-1])["persistent"] == 1
    gbk.gbk_survey_set_tuning(geoms, None)
    assert gbk.gbk_survey_get_tuning(geoms) == t
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_set_tuning(geoms, 1, 0, 512)
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_set_tuning(geoms, 1, cs, 300)
    with pytest.raises(gbk.GbkError):
        gbk.gbk_survey_set_tuning(geoms, 2, cs, 512)
    big = SINGLE_GEOM.with_(nx=160, ny=160, nz=64)
    assert gbk.gbk_survey_get_tuning(geoms + [big])["cluster_ctas"] > cs
    with pytest.raises(gbk.GbkError):  # a 1-CTA cluster cannot hold a 160 x 160 galaxy's rows
        gbk.gbk_survey_set_tuning(geoms + [big], 1, 1, 512)
    # the table size does not depend on the launch shape
    tables = gbk.gbk_survey_workspace_bytes(geoms)
    gbk.gbk_survey_set_tuning(geoms, 0)
    assert gbk.gbk_survey_workspace_bytes(geoms) == tables
    gbk.gbk_survey_set_tuning(geoms, None)
