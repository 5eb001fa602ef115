"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one of them.

Each mutant is a one-expression edit of ``oracle/gbk_oracle.c`` (a dropped
term, a wrong sign, a wrong constant, an off-by-one), compiled on the CPU into
a temporary library.  No mutant reads or writes outside its buffers.
"""
import os
import subprocess

import pytest

import oracle
from oracle_pins import ALL_PINS

SRC = os.path.join(os.path.dirname(oracle.__file__), "gbk_oracle.c")

MUTANTS = [
    ("eq1_sign", "double xe = -dx * sin(pa) + dy * cos(pa);", "double xe = dx * sin(pa) + dy * cos(pa);"),
    ("eq1_sin_cos_swapped", "double xe = -dx * sin(pa) + dy * cos(pa);", "double xe = -dx * cos(pa) + dy * sin(pa);"),
    ("eq2_sign", "double ye = -dx * cos(pa) - dy * sin(pa);", "double ye = -dx * cos(pa) + dy * sin(pa);"),
    ("eq3_no_deprojection", "double yd = ye / cos(inc);", "double yd = ye;"),
    ("eq3_cos_as_sin", "double yd = ye / cos(inc);", "double yd = ye / sin(inc);"),
    ("eq5_scale_inverted", "exp(-r / p[OG_H])", "exp(-r * p[OG_H])"),
    ("eq6_missing_2_over_pi", "return (2.0 / OG_PI) * p[OG_VMAX] * atan(r / p[OG_RT]) / r;",
     "return p[OG_VMAX] * atan(r / p[OG_RT]) / r;"),
    ("eq6_rt_inverted", "atan(r / p[OG_RT]) / r;", "atan(r * p[OG_RT]) / r;"),
    ("eq8_cos_i", "*sin_i = sin(inc);", "*sin_i = cos(inc);"),
    ("eq7_a_g_swapped", "pow(q, p[OG_H]) / (1.0 + pow(q, p[OG_I0]))", "pow(q, p[OG_I0]) / (1.0 + pow(q, p[OG_H]))"),
    ("eq7_one_dropped", "pow(q, p[OG_H]) / (1.0 + pow(q, p[OG_I0]))", "pow(q, p[OG_H]) / pow(q, p[OG_I0])"),
    ("eq7_rt_inverted", "double q = r / p[OG_RT];", "double q = r * p[OG_RT];"),
    ("eq7_centre_undefined", "if (!(r > 0.0)) return 0.0;", "if (!(r > 0.0)) return NAN;"),
    ("vfield_sigma_model_dropped", "maps[2 * np + s] = p[OG_SIG0];", "maps[2 * np + s] = 0.0;"),
    ("vfield_curve_ignored", "og_vrot_over_r(g->model == 2, p, r)", "og_vrot_over_r(0, p, r)"),
    ("eq8_degrees", "double inc = p[OG_INCL] * OG_PI / 180.0;", "double inc = p[OG_INCL];"),
    ("line_width_sqrt2", "ext[(size_t)ze * d.exf * d.eyf + i] = br[i] * norm * exp(-0.5 * t * t);",
     "ext[(size_t)ze * d.exf * d.eyf + i] = br[i] * norm * exp(-t * t);"),
    ("line_norm_dropped_sigma", "double norm = g->dv / (s * sqrt(2.0 * OG_PI));",
     "double norm = g->dv / sqrt(2.0 * OG_PI);"),
    ("channel_grid_off_by_half", "return g->vc + (kc - 0.5 * (g->nz - 1)) * g->dv;",
     "return g->vc + (kc - 0.5 * g->nz) * g->dv;"),
    ("fine_pixel_centre", "double y = ((double)(ye - d.rxy) + 0.5) / d.u - 0.5;",
     "double y = ((double)(ye - d.rxy)) / d.u;"),
    ("mode_b_linear_sum", "return sqrt(p[OG_SIG0] * p[OG_SIG0] + sl * sl);", "return p[OG_SIG0] + sl;"),
    ("taps_unnormalised", "for (int j = 0; j <= 2 * R; ++j) w[j] /= s;", "for (int j = 0; j <= 2 * R; ++j) w[j] /= 1.0;"),
    ("taps_sigma_sqrt2", "w[j + R] = exp(-(double)j * (double)j / (2.0 * sigma * sigma));",
     "w[j + R] = exp(-(double)j * (double)j / (sigma * sigma));"),
    ("radius_floor", "return (int)ceil(halo * sigma);", "return (int)floor(halo * sigma);"),
    ("lsf_sigma_not_in_channels", "d->sig_z = u * (g->lsf_fwhm / OG_FWHM_PER_SIGMA) / g->dv;",
     "d->sig_z = u * (g->lsf_fwhm / OG_FWHM_PER_SIGMA);"),
    ("fwhm_as_sigma", "d->sig_xy = u * g->psf_fwhm / OG_FWHM_PER_SIGMA;", "d->sig_xy = u * g->psf_fwhm / 2.0;"),
    ("moment2_no_sqrt", "maps[2 * np + s] = sqrt(s2 / s0);", "maps[2 * np + s] = s2 / s0;"),
    ("moment1_unnormalised", "double m1 = s1 / s0;", "double m1 = s1;"),
    ("moment_invalid_ignored", "if (!(s0 > OG_INVALID_FRACTION * scale)) {", "if (0) {"),
    ("downsample_sum", "coarse[((size_t)k * ny + j) * nx + i] = acc * inv;", "coarse[((size_t)k * ny + j) * nx + i] = acc;"),
    ("chi2_weight_dropped", "rv = (double)w_v[s] * (maps[np + s] - (double)v_obs[s]);",
     "rv = (maps[np + s] - (double)v_obs[s]);"),
    ("chi2_mask_ignored", "if (mask[s] != 0 && maps[s] > 0.0) {", "if (maps[s] > 0.0) {"),
    ("chi2_dispersion_term_dropped", "og_add(&acc, rs * rs);", "(void)rs;"),
    ("parameter_domain_dropped", "int ok = p[OG_INCL] >= 0.0 && p[OG_INCL] < 90.0 && p[OG_RT] > 0.0;", "int ok = 1;"),
    ("inclination_domain_closed", "p[OG_INCL] < 90.0 && p[OG_RT] > 0.0;", "p[OG_INCL] <= 90.0 && p[OG_RT] > 0.0;"),
]


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutant %s: pattern not unique" % name
    msrc = tmp_path / ("m_%s.c" % name)
    msrc.write_text(src.replace(old, new))
    lib = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", str(msrc), "-o", str(lib), "-lm"],
                   check=True, capture_output=True)
    return str(lib)


def _caught(lib_path):
    oracle.use_library(lib_path)
    failed = []
    for pin in ALL_PINS:
        try:
            pin(oracle)
        except Exception:
            failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    path = _build(tmp_path, name, old, new)
    try:
        failed = _caught(path)
    finally:
        oracle.use_library(oracle.build.build())
    assert failed, "mutant %s survived every pin" % name
