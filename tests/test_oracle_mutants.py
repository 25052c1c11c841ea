"""Planted mistakes in the CPU oracle must each fail at least one pin.

Each mutant is a copy of ``oracle/splotch_oracle.c`` with one plausible slip
(a dropped term, a wrong sign, index or operand), compiled on the CPU and run
through every pin of ``oracle_pins``.  A mutant that passes all pins would
mean the pins cannot tell that mistake from the real oracle.
"""
import os
import tempfile

import pytest

import oracle
import oracle_pins

MUTANTS = {
    "y_sign": ("float Y = cy - (F * yc) / zc;", "float Y = cy + (F * yc) / zc;"),
    "full_fov": ("tan(fov_deg * (M_PI / 360.0))", "tan(fov_deg * (M_PI / 180.0))"),
    "focal_from_width": ("(0.5 * (double)H) / tan", "(0.5 * (double)W) / tan"),
    "left_handed": ("cross3(f, up, s0);", "cross3(up, f, s0);"),
    "up_flipped": ("cross3(s, f, u);", "cross3(f, s, u);"),
    "translation_sign": ("m[4 * r + 3] = (float)(-dot3(rows[r], eye));",
                         "m[4 * r + 3] = (float)(dot3(rows[r], eye));"),
    "radius_no_depth": ("float r = (F * h) / zc;", "float r = F * h;"),
    "radius_no_floor": ("if (!(R > rmin)) R = rmin;", ""),
    "near_plane_ignored": ("if (!(zc > zn) || !(zc <= zf)) return;", "if (!(zc > 0.0f) || !(zc <= zf)) return;"),
    "far_plane_exclusive": ("if (!(zc > zn) || !(zc <= zf)) return;", "if (!(zc > zn) || !(zc < zf)) return;"),
    "far_plane_ignored": ("if (!(zc > zn) || !(zc <= zf)) return;", "if (!(zc > zn)) return;"),
    "box_too_narrow": ("int i0 = (int)ceilf(xl) - 1, i1 = (int)floorf(xh) + 1;",
                       "int i0 = (int)ceilf(xl) + 1, i1 = (int)floorf(xh) - 1;"),
    "coverage_wrong_operand": ("float d2 = dx * dx + dy * dy;", "float d2 = dx * dx + dx * dy;"),
    "sigma_equals_R": ("double sg = sor * (double)o->R;", "double sg = (double)o->R;"),
    "gaussian_half_exponent": ("return exp(-(dx * dx + dy * dy) / (sg * sg));",
                               "return exp(-(dx * dx + dy * dy) / (2.0 * sg * sg));"),
    "colour_next_entry_dropped": ("tau * (double)cmap[3 * (k + 1) + c]", "tau * (double)cmap[3 * k + c]"),
    "colour_scale_n": ("double f = It * (double)(n - 1);", "double f = It * (double)n;"),
    "brightness_dropped": ("e[c] = beta * ((1.0 - tau)", "e[c] = 1.0 * ((1.0 - tau)"),
    "tile_half_side": ("float hd = 0.70710677f * (float)T;", "float hd = 0.25f * (float)T;"),
    "tile_corner_not_centre": ("float cx = ((float)tx + 0.5f) * (float)T;", "float cx = (float)tx * (float)T;"),
    "tile_rule_no_support": ("float thr = o->R + hd;", "float thr = hd;"),
    "rt_depth_front_first": ("if (za != zb) return za > zb ? -1 : 1;", "if (za != zb) return za > zb ? 1 : -1;"),
    "rt_depth_one_species": ("const double st = absorb[type_of(&s, k)];", "const double st = absorb[0];"),
    "rt_depth_emission_over_absorption_dropped": ("v[c] = v[c] * t + (E / A) * (1.0 - t);",
                                                  "v[c] = v[c] * t + (1.0 - t);"),
    "rt_map_alpha_not_multiplied": ("if (Amap) Amap[3 * ((size_t)b * nx + a) + c] *= t;",
                                    "if (Amap) Amap[3 * ((size_t)b * nx + a) + c] = t;"),
    "vector_colour_ignored": ("if (s->vec && s->vec[t])", "if (0 && s->vec)"),
    "vector_components_swapped": ("for (int c = 0; c < 3; ++c) e[c] = beta * rgb[c];",
                                  "for (int c = 0; c < 3; ++c) e[c] = beta * rgb[2 - c];"),
    "image_transposed": ("double *q = &a[3 * ((size_t)j * W + i)];\n                    for (int c = 0; c < 3; ++c) q[c] += e[k][c] * w;",
                         "double *q = &a[3 * ((size_t)(i % H) * W + (j % W))];\n                    for (int c = 0; c < 3; ++c) q[c] += e[k][c] * w;"),
    "final_wrong": ("O[i] = -expm1(-a[i]);", "O[i] = 1.0 - exp(-2.0 * a[i]);"),
    "normalise_wrong_origin": ("(out[i] - i_min) / span", "(out[i] - i_max) / span"),
    "log_dropped": ("out[i] = i_log ? log(v > 1e-30 ? v : 1e-30) : v;", "out[i] = v;"),
    "quantise_truncates": ("double r = rint(a / q) * q;", "double r = floor(a / q) * q;"),
    "species_off_by_one": ("while (t + 1 < s->n_types && i >= s->type_begin[t + 1]) ++t;",
                           "while (t + 1 < s->n_types && i > s->type_begin[t + 1]) ++t;"),
}


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, workdir):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    lib = oracle.build_variant(src.replace(old, new), os.path.join(workdir, f"mut_{name}.so"))
    failed = []
    with oracle.using(lib):
        for pin in oracle_pins.ALL_PINS:
            try:
                pin()
            except Exception:  # AssertionError or a rejected call: the pin noticed
                failed.append(pin.__name__)
    assert failed, f"no pin catches mutant {name}"
