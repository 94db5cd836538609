"""The oracle's pins catch plausible mistakes.

Each case copies lp_oracle.c, plants one mistake of the kind a transcription
of the paper could make (a dropped term, a wrong sign or index, a transposed
operand, a changed tie rule or constant), compiles the copy, and runs the pins
that guard that function against it: at least one must fail.  The unmodified
copy, compiled the same way, passes every one of those pins.
"""
import math
import os

import pytest

import oracle
import test_oracle_describe as DS
import test_oracle_detect as D
import test_oracle_hard_bins as HB
import test_oracle_literal as L
import test_oracle_match_ransac as MR
import test_oracle_mlp as ML
import test_oracle_mosaic as MO
import test_oracle_rigid as R

SRC = os.path.join(os.path.dirname(oracle.__file__), "lp_oracle.c")


def _orient_ramps():
    for img, want in (("row", 0), ("col", 9), ("negcol", 27), ("diag", 4), ("negrow", 18)):
        DS.test_orient_ramps(img, want)


def _detect_brute():
    D.test_detect_bruteforce((16, 16), (2, 4, 8, 16), 256)
    D.test_detect_bruteforce((13, 17), (3, 4), 4)


def _rigid_exact():
    for th in (0.3, -1.2, 2.9, math.pi / 2):
        R.test_rigid_fit_recovers_exact_transform(th)


def _border():
    L.test_border_rejection_keeps_exactly_clamp_free_points(False)
    L.test_border_rejection_keeps_exactly_clamp_free_points(True)


def _finite_alpha():
    for a in (1e-6, 0.02, 3.0):
        L.test_finite_alpha_ramp_is_eq1(a)


# (name, text in lp_oracle.c, planted text, pins guarding it)
MUTANTS = [
    ("gray_rounding_term_dropped",
     "114u * p[2] + 500u;", "114u * p[2];",
     [D.test_gray_exact_rational, D.test_gray_axis_and_extremes]),
    ("gray_red_green_swapped",
     "299u * p[0] + 587u * p[1]", "299u * p[1] + 587u * p[0]",
     [D.test_gray_exact_rational, D.test_gray_axis_and_extremes]),
    ("detect_tie_takes_first_index",
     "return g1 > g2 || (g1 == g2 && i1 > i2);", "return g1 > g2 || (g1 == g2 && i1 < i2);",
     [D.test_detect_constant_image_ramp_tiebreak, _detect_brute]),
    ("detect_literal_ramp_sign",
     "double v = (double)g + alpha * (double)(r + 1);", "double v = (double)g - alpha * (double)(r + 1);",
     [D.test_detect_literal_alpha_equals_limit, _finite_alpha]),
    ("keypoints_one_per_window",
     "K += 2 * (int64_t)(H / Ls[l]) * (int64_t)(W / Ls[l]);", "K += (int64_t)(H / Ls[l]) * (int64_t)(W / Ls[l]);",
     [D.test_num_keypoints_closed_form]),
    ("region_exponent_sign",
     "pow((double)Ls[l] / (double)Lmax, -0.5)", "pow((double)Ls[l] / (double)Lmax, 0.5)",
     [D.test_region_ws_closed_form]),
    ("region_truncated",
     "int w = (int)floor(beta * (double)Ls[l] + 0.5);", "int w = (int)floor(beta * (double)Ls[l]);",
     [D.test_region_ws_closed_form]),
    ("orient_weight_truncated",
     "return (uint32_t)floor(65536.0 * sqrt((double)s) + 0.5);", "return (uint32_t)floor(65536.0 * sqrt((double)s));",
     [DS.test_orient_weight_exhaustive_integer_bracket]),
    ("orient_bin_operands_transposed",
     "double phi = atan2((double)b, (double)a);", "double phi = atan2((double)a, (double)b);",
     [DS.test_orient_bin_exhaustive]),
    ("orient_row_gradient_sign",
     "int a = px(gray, H, W, pitch, yy + 1, xx) - px(gray, H, W, pitch, yy - 1, xx);",
     "int a = px(gray, H, W, pitch, yy - 1, xx) - px(gray, H, W, pitch, yy + 1, xx);",
     [_orient_ramps]),
    ("orient_tie_takes_last_bin",
     "if (h[j] > h[best]) best = j;", "if (h[j] >= h[best]) best = j;",
     [DS.test_orient_exact_tie_lowest_bin_wins]),
    ("describe_clamp_dropped",
     "if (q > 0.2) q = 0.2;", "if (q > 2.0) q = 2.0;",
     [DS.test_describe_ramp_closed_forms]),
    ("describe_column_gradient_sign",
     "double b = bil(gray, H, W, pitch, py - s, pxx + c) - bil(gray, H, W, pitch, py + s, pxx - c);",
     "double b = bil(gray, H, W, pitch, py + s, pxx - c) - bil(gray, H, W, pitch, py - s, pxx + c);",
     [DS.test_describe_ramp_closed_forms, DS.test_describe_upright_equals_integer_eq5]),
    ("describe_cells_transposed",
     "int cell = ((u + R) / s_) * 4 + (v + R) / s_;", "int cell = ((v + R) / s_) * 4 + (u + R) / s_;",
     [DS.test_describe_upright_equals_integer_eq5]),
    ("describe_soft_split_swapped",
     "h[cell * 8 + b0] += m * (1.0 - t);", "h[cell * 8 + b0] += m * t;",
     [DS.test_describe_ramp_closed_forms]),
    ("hard_edge_to_lower_sector",
     "if (b >= 0 && a > 0) return b < a ? 0 : 1;", "if (b >= 0 && a > 0) return b <= a ? 0 : 1;",
     [HB.test_octant_edges_and_interiors, HB.test_octant_matches_atan2_sector_away_from_edges]),
    ("hard_sectors_2_3_swapped",
     "if (a <= 0 && b > 0) return b > -a ? 2 : 3;", "if (a <= 0 && b > 0) return b > -a ? 3 : 2;",
     [HB.test_describe_hard_ramp_closed_forms]),
    ("hard_sector_operands_transposed",
     "h[cell * 8 + or_octant(a, b)] +=", "h[cell * 8 + or_octant(b, a)] +=",
     [HB.test_describe_hard_ramp_closed_forms, HB.test_describe_hard_upright_equals_integer_eq5]),
    ("hard_fx_weights_transposed",
     "int64_t top = v00 * (2048 - fc) + v01 * fc;\n    int64_t bot = v10 * (2048 - fc) + v11 * fc;",
     "int64_t top = v00 * (2048 - fr) + v01 * fr;\n    int64_t bot = v10 * (2048 - fr) + v11 * fr;",
     [HB.test_describe_hard_ramp_closed_forms]),
    ("hard_fx_turn_sign",
     "int64_t pr = (int64_t)u * cq - (int64_t)v * sq,", "int64_t pr = (int64_t)u * cq + (int64_t)v * sq,",
     [HB.test_describe_hard_ramp_closed_forms, HB.test_describe_hard_rotation_90_invariant]),
    ("hard_turn_truncated",
     "*cq = (int)floor(2048.0 * cos(th) + 0.5);", "*cq = (int)floor(2048.0 * cos(th));",
     [HB.test_turn_table_is_rounded_2048_cos_sin]),
    ("describe_turn_sign",
     "double py = y + u * c - v * s;", "double py = y + u * c + v * s;",
     [DS.test_describe_ramp_closed_forms, DS.test_describe_rotation_90_invariant]),
    ("border_radius_short",
     "const int P = (int)ceil(2.0 * sqrt(2.0) * ws[k] + 1.5) + 1;",
     "const int P = (int)ceil(2.0 * sqrt(2.0) * ws[k] + 1.5);",
     [_border]),
    ("match_ratio_not_squared",
     "b1 < ratio * ratio * b2", "b1 < ratio * b2",
     [MR.test_match_vs_numpy_bruteforce]),
    ("match_tie_takes_last_index",
     "if (e < b1) {", "if (e <= b1) {",
     [MR.test_match_exact_tie_takes_the_lowest_index]),
    ("match_without_ratio_needs_two",
     ": nbv >= 1;", ": nbv >= 2;",
     [L.test_match_without_ratio_test_is_the_nearest_neighbour]),
    ("philox_key_constant",
     "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE87u;",
     [MR.test_philox_known_answers]),
    ("philox_words_swapped",
     "c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;", "c0 = n0; c1 = lo0; c2 = n2; c3 = lo1;",
     [MR.test_philox_known_answers]),
    ("dlt_row_sign",
     "double r1[9] = {0, 0, 0, x, y, 1, -x * yp, -y * yp, yp};",
     "double r1[9] = {0, 0, 0, x, y, 1, -x * yp, -y * yp, -yp};",
     [MR.test_dlt4_exact_and_square_to_quad]),
    ("denormalise_operands_transposed",
     "mat3_mul(Hn, Ts, t);", "mat3_mul(Ts, Hn, t);",
     [MR.test_dlt4_exact_and_square_to_quad]),
    ("refit_second_row_dropped",
     "AtA[9 * j + k] += r0[j] * r0[k] + r1[j] * r1[k];", "AtA[9 * j + k] += r0[j] * r0[k];",
     [MR.test_refit_equals_numpy_svd]),
    ("refit_eigenvector_transposed",
     "for (int j = 0; j < 9; ++j) h[j] = V[9 * j + 0];", "for (int j = 0; j < 9; ++j) h[j] = V[j];",
     [MR.test_refit_equals_numpy_svd]),
    ("score_accepts_w_negative",
     "        int in = 0;\n        if (w > 0) {", "        int in = 0;\n        if (w != 0) {",
     [MR.test_score_counts_and_w_nonpositive]),
    ("score_boundary_inclusive",
     "in = u * u + v * v < t2;", "in = u * u + v * v <= t2;",
     [MR.test_score_counts_and_w_nonpositive]),
    ("ransac_tie_takes_latest",
     "        if (c > bestc) {\n            bestc = c;\n            *best_t = t;\n            memcpy(Hb, Ht, sizeof Hb);\n"
     "        }\n    }\n    if (bestc < 0) return 1;",
     "        if (c >= bestc) {\n            bestc = c;\n            *best_t = t;\n            memcpy(Hb, Ht, sizeof Hb);\n"
     "        }\n    }\n    if (bestc < 0) return 1;",
     [MR.test_ransac_best_is_earliest_max]),
    ("rigid_sine_sign",
     "Ss += ax * by - ay * bx;", "Ss += ay * bx - ax * by;",
     [_rigid_exact]),
    ("rigid_translation_sign",
     "H[2] = cxb - (c * cxa - sn * cya);", "H[2] = cxb - (c * cxa + sn * cya);",
     [_rigid_exact]),
    ("mlp_relu_derivative_dropped",
     "d2[j] = h2[j] > 0 ? dz * w3[j] : 0;", "d2[j] = dz * w3[j];",
     [ML.test_loss_gradient_matches_central_differences]),
    ("mlp_input_gradient_reversed",
     "gW1[8 * i + j] += d1[i] * xn[j];", "gW1[8 * i + j] += d1[i] * xn[7 - j];",
     [ML.test_loss_gradient_matches_central_differences]),
    ("adam_bias_correction_dropped",
     "params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);", "params[i] -= lr * m[i] / (sqrt(v[i]) + eps);",
     [ML.test_adam_first_step_closed_form]),
    ("guided_floor_dropped",
     "if (!(p > lo)) p = lo;", "if (p < 0) p = lo;",
     [ML.test_guided_weights_are_exact_integers]),
    ("guided_stop_bound",
     "return r <= 0.01;", "return r <= 0.05;",
     [ML.test_guided_stop_is_the_standard_bound]),
    ("feature_angle_wrap",
     "if (dth >= 180.0) dth -= 360.0;", "if (dth > 180.0) dth -= 360.0;",
     [ML.test_features_by_hand]),
    ("orient_window_one_sided",
     "for (int u = -R; u <= R; ++u)", "for (int u = -R; u < R; ++u)",
     [DS.test_orient_rotation_90_histogram_roll, DS.test_orient_exact_tie_lowest_bin_wins]),
    ("bilinear_wrong_fraction",
     "double top = v00 + fc * (v01 - v00);", "double top = v00 + fr * (v01 - v00);",
     [DS.test_describe_ramp_closed_forms, DS.test_describe_rotation_90_invariant]),
    ("describe_second_normalisation_dropped",
     "for (int j = 0; j < 128; ++j) out[j] /= n2;", "for (int j = 0; j < 128; ++j) out[j] /= 1.0;",
     [DS.test_describe_unit_norm_and_invalid, DS.test_describe_ramp_closed_forms]),
    ("match_distance_not_rooted",
     "d1[q] = sqrt(b1);", "d1[q] = b1;",
     [MR.test_match_vs_numpy_bruteforce]),
    ("sample_duplicates_kept",
     "(uint64_t)M) >> 32);\n        int dup = 0;\n        for (int q = 0; q < n; ++q) dup |= idx[q] == i;",
     "(uint64_t)M) >> 32);\n        int dup = 0;\n        for (int q = 0; q < n; ++q) dup |= 0;",
     [MR.test_ransac_sample_distinct_uniform]),
    ("jacobi_rotation_sign",
     "a[k][p] = c * akp - s * akq;", "a[k][p] = c * akp + s * akq;",
     [MR.test_eig_sym_vs_numpy, MR.test_refit_equals_numpy_svd]),
    ("rigid_centroid_variable",
     "cxb = sxb / n, cyb = syb / n;", "cxb = sxa / n, cyb = syb / n;",
     [_rigid_exact]),
    ("mlp_first_bias_dropped",
     "double s = b1[i];", "double s = 0;",
     [ML.test_closed_form_networks, ML.test_loss_gradient_matches_central_differences]),
    ("mlp_distance_ratio_inverted",
     "f[0] = d2[i] > 0 ? d1[i] / d2[i] : 1.0;", "f[0] = d1[i] > 0 ? d2[i] / d1[i] : 1.0;",
     [ML.test_features_by_hand]),
    ("adam_second_moment_not_squared",
     "v[i] = b2 * v[i] + (1 - b2) * grad[i] * grad[i];", "v[i] = b2 * v[i] + (1 - b2) * fabs(grad[i]);",
     [ML.test_adam_first_step_closed_form]),
    ("guided_support_floor_dropped",
     "stop = or_guided_stop_k(s_in, prefix[M - 1], Tg, k) && bestc >= (int64_t)min_support &&",
     "stop = or_guided_stop_k(s_in, prefix[M - 1], Tg, k) &&",
     [ML.test_ransac_prior_support_floor]),
    ("guided_plain_fraction_bound_dropped",
     "(int64_t)min_support &&\n               or_guided_stop_k((uint64_t)bestc, (uint64_t)M, Tg, k);",
     "(int64_t)min_support;",
     [ML.test_ransac_prior_support_floor]),
    ("guided_weight_truncated",
     "acc += (uint64_t)floor(65536.0 * p + 0.5);", "acc += (uint64_t)floor(65536.0 * p);",
     [ML.test_guided_weights_are_exact_integers]),
    ("border_right_edge_loose",
     "x + P > W - 1 || y + P > H - 1", "x + P > W || y + P > H - 1",
     [_border]),
    ("region_default_beta_inverted",
     "beta0 = sqrt((double)Lmin / (double)Lmax) / (double)d;", "beta0 = sqrt((double)Lmax / (double)Lmin) / (double)d;",
     [D.test_region_ws_closed_form]),
    ("render_mean_truncated",
     "(uint8_t)floor(sum[c] / n + 0.5) : 0;", "(uint8_t)floor(sum[c] / n) : 0;",
     [MO.test_render_half_pixel_shift_is_the_mean_of_neighbours, MO.test_render_identity_and_integer_overlap]),
    ("render_vertical_fraction",
     "sum[c] += top + fv * (bot - top);", "sum[c] += top + fu * (bot - top);",
     [MO.test_render_half_pixel_shift_is_the_mean_of_neighbours, MO.test_render_identity_and_integer_overlap]),
    ("mosaic_reference_tie_takes_last",
     "if (ref < 0 || deg[i] > deg[ref]) { ref = i; via = link; }",
     "if (ref < 0 || deg[i] >= deg[ref]) { ref = i; via = link; }",
     [MO.test_degree_tie_takes_the_lowest_index, MO.test_chain_graph_rounds_and_references]),
    ("mosaic_entry_direction",
     "if (pairs[2 * q] == from) { memcpy(M, HM + 9 * q, sizeof(double) * 9); return 0; }",
     "if (pairs[2 * q] != from) { memcpy(M, HM + 9 * q, sizeof(double) * 9); return 0; }",
     [MO.test_star_graph_is_one_round, MO.test_chain_graph_rounds_and_references,
      MO.test_disconnected_image_stays_unplaced_and_canvas_box]),
]

ALL_PINS = []
for _, _, _, _pins in MUTANTS:
    for _p in _pins:
        if _p not in ALL_PINS:
            ALL_PINS.append(_p)


def _source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_copy_passes_every_pin(tmp_path):
    so = oracle.compile_variant(_source(), str(tmp_path / "orig.so"))
    with oracle.use_library(so):
        for pin in ALL_PINS:
            pin()


@pytest.mark.parametrize("name,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, old, new, pins):
    src = _source()
    assert src.count(old) == 1, f"{name}: the text to plant into is not unique in lp_oracle.c"
    so = oracle.compile_variant(src.replace(old, new), str(tmp_path / f"{name}.so"))
    failed = []
    with oracle.use_library(so):
        for pin in pins:
            try:
                pin()
            except Exception:       # an assertion, or an error the wrong result raises
                failed.append(pin.__name__)
    assert failed, f"no pin caught {name}"
