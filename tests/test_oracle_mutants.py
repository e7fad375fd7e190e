"""Plants plausible mistakes in copies of oracle.c (on the CPU) and checks
that the pins of _pins.py catch every one: a dropped term, a wrong sign, a
wrong index, a transposed operand, an off-by-one, a lost clamp, ..."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "bounds_min_as_max": ("if (p < lo[a]) lo[a] = p;", "if (p > lo[a]) lo[a] = p;"),
    "bounds_negative_zero_kept": ("        lo[a] = lo[a] + 0.0f;\n", ""),
    "bounds_index_off_by_one": ("(int64_t)vi >= nverts", "(int64_t)vi > nverts"),
    "plan_floor_not_ceil": ("double r = ceil((double)e[a] * k);", "double r = floor((double)e[a] * k);"),
    "plan_sqrt_not_cbrt": ("(d == 3) ? cbrt(q)", "(d == 3) ? sqrt(q)"),
    "plan_scale_inverted": ("scale[a] = (float)res[a] / e[a];", "scale[a] = e[a] / (float)res[a];"),
    "plan_flat_axis_counted": ("if (n > 0 && e[a] > 0.0f) { ++d;", "if (n > 0) { ++d;"),
    "cell_sign": ("float t = p - lo;", "float t = p + lo;"),
    "cell_no_clamp_hi": ("if (f > (float)(res - 1)) return res - 1;", "if (f > (float)res) return res - 1;"),
    "count_exclusive_hi": ("cnt *= (int64_t)(ch - cl + 1);", "cnt *= (int64_t)(ch - cl) + (ch == cl);"),
    "box_hi_from_min": ("if (k == 0 || p > bh) bh = p;", "if (k == 0 || p < bh) bh = p;"),
    "scan_inclusive": ("offsets[i] = s;\n        s += V[i];", "s += V[i];\n        offsets[i] = s;"),
    "markers_from_zero": ("for (int64_t i = 1; i < n; ++i) O[offsets[i]] = 1;",
                          "for (int64_t i = 0; i < n; ++i) O[offsets[i]] = 1;"),
    "segment_no_reset": ("if (j == 0 || O[j] != O[j - 1]) run = 0;", "if (j == 0) run = 0;"),
    "coords_wrong_divisor": ("int64_t y = (rid - z * mx * my) / mx;", "int64_t y = (rid - z * mx * my) / my;"),
    "coords_x_y_swapped": ("out[0] = lo[0] + (int32_t)x;\n    out[1] = lo[1] + (int32_t)y;",
                           "out[0] = lo[0] + (int32_t)y;\n    out[1] = lo[1] + (int32_t)x;"),
    "linear_wrong_index": ("(int64_t)res[1] * (int64_t)g[2]", "(int64_t)res[0] * (int64_t)g[2]"),
    "sort_unstable_desc": ("return a->j < b->j ? -1 : (a->j > b->j ? 1 : 0);",
                           "return a->j > b->j ? -1 : (a->j < b->j ? 1 : 0);"),
    "ranges_inclusive": ("int64_t v = g[c];\n        G[c] = (int32_t)s;\n        s += v;",
                         "int64_t v = g[c];\n        s += v;\n        G[c] = (int32_t)s;"),
    "cell_scale_dropped": ("float u = t * scale;", "float u = t;"),
    "cell_nan_not_zero": ("if (isnan(u)) return 0;\n    float f = floorf(u);", "float f = ceilf(u) - 1.0f;"),
    "counting_exclusive_scan_shift": ("cnt[c] = s;\n        G[c] = (int32_t)s;\n        s += v;\n    }\n    for (int64_t i = 0;",
                                      "cnt[c] = s + v - v;\n        G[c] = (int32_t)(s + (c > 0));\n        s += v;\n    }\n    for (int64_t i = 0;"),
    # culling mode
    "cull_normal_axis_dropped": ("for (int s = 0; s < 10; ++s) {", "for (int s = 1; s < 10; ++s) {"),
    "cull_center_at_corner": ("(float)x + 0.5f, (float)y + 0.5f", "(float)x, (float)y + 0.5f"),
    "cull_negative_slack": ("const float R = 0.5f * S + S * t;", "const float R = 0.5f * S - S * t;"),
    "cull_radius_doubled": ("const float R = 0.5f * S + S * t;", "const float R = S + S * t;"),
    "cull_edge_axis_sign": ("ax[1 + j][1] = -e[j][2];", "ax[1 + j][1] = e[j][2];"),
    "cull_missing_edge": ("e[1][a] = q[6 + a] - q[3 + a];", "e[1][a] = q[6 + a] - q[a];"),
    "cull_pmax_from_min": ("if (k == 0 || p > pmax) pmax = p;", "if (k == 0 || p < pmax) pmax = p;"),
    "cull_last_vertex_skipped": ("for (int k = 0; k < 3; ++k) {\n            float p = a[0]",
                                 "for (int k = 0; k < 2; ++k) {\n            float p = a[0]"),
    "cull_normal_component_swapped": ("ax[0][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];",
                                      "ax[0][1] = e[0][0] * e[1][2] - e[0][2] * e[1][0];"),
    "cull_no_far_face_clamp": ("q[3 * v + a] = u > (float)res[a] ? (float)res[a] : u;", "q[3 * v + a] = u;"),
    # plan and mapping
    "plan_no_res_max_clamp": ("if (r > (double)OR_RES_MAX) r = (double)OR_RES_MAX;", ""),
    "plan_overflow_unchecked": ("if (nc > INT32_MAX) return OR_EOVERFLOW;", ""),
    "plan_cbrt_for_two_axes": ("(d == 2) ? sqrt(q)", "(d == 2) ? cbrt(q)"),
    "plan_volume_in_fp32": ("vol = vol * (double)e[a];", "vol = (double)(float)(vol * (double)e[a]);"),
    "cell_no_clamp_lo": ("if (f < 0.0f) return 0;", ""),
    "scan_overflow_unchecked": ("if (s > INT32_MAX) { *total = s; return OR_EOVERFLOW; }", ""),
    "coords_z_divisor": ("int64_t z = rid / (mx * my);", "int64_t z = rid / (mx * mx);"),
    "coords_x_term": ("int64_t x = rid - mx * (y + my * z);", "int64_t x = rid - mx * (y + mx * z);"),
    "inclusive_sum_dropped_term": ("O[j] = O[j] + O[j - 1];", "O[j] = O[j - 1];"),
    "place_reversed": ("for (int64_t j = 0; j < NO; ++j) refs[cnt[C[j]]++] = O[j];",
                       "for (int64_t j = NO - 1; j >= 0; --j) refs[cnt[C[j]]++] = O[j];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "oracle_mut.c"
    mut.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mut), str(tmp_path / "liboracle_mut.so"))
    code = ("import sys; sys.path[:0] = [%r, %r]\n"
            "import oracle; oracle.use_library(%r)\n"
            "import _pins; f = _pins.run_all(); print(f); sys.exit(1 if f else 0)\n") % (ROOT, HERE, lib)
    # a mutant may also crash (an out-of-range cell id): that counts as caught
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived every pin:\n{r.stdout}\n{r.stderr}"
