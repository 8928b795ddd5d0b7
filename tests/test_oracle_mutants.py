"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's source -- a flipped
sign, a dropped factor, a wrong exponent, index or bound, a transposed
operand, a skipped step -- and runs the pins named beside it against that
copy in a child pytest: for the C source (MUTANTS) a build made with the
oracle's own compiler flags, loaded through PPMD_ORACLE_LIB; for the NumPy
network (MLP_MUTANTS) the copy imported as `oracle.mlp`, for the
package's own Python (PKG_MUTANTS) a copy of the package imported as
`oracle`, and for the classifier parity tests' comparison helpers
(PIPE_MUTANTS) a copy imported as `oracle_pipeline`, before the pins are
collected.  A case passes when at least one of its pins fails, so every
entry records which pin stands guard over which part of the oracle.  The
CUDA library is not involved.
"""
import os
import shutil
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ppmd_oracle.c")
MD = "tests/test_oracle_md.py::"
AN = "tests/test_oracle_analysis.py::"
BF = "tests/test_oracle_mlp_bf16.py::"
MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")
PKG_SRC = os.path.join(ROOT, "oracle", "__init__.py")

# name: (text of the oracle, the mistake, which occurrence (0 = first), pins)
MUTANTS = {
    # periodic domain and cells (Sec. 3.5)
    "wrap_by_rint": ("double y = x - L * floor(x / L);", "double y = x - L * rint(x / L);", 0,
                     [MD + "test_vv_wraps_into_box"]),
    "min_image_by_floor": ("t = t - L[d] * rint(t / L[d]);", "t = t - L[d] * floor(t / L[d]);", 0,
                           [MD + "test_lattice_energy_closed_form"]),
    "cell_index_transposed": ("cell_of[i] = (cz * nc[1] + cy) * nc[0] + cx;",
                              "cell_of[i] = (cx * nc[1] + cy) * nc[0] + cz;", 0,
                              [MD + "test_cells_contain_their_atoms"]),
    "stencil_misses_a_layer": ("for (int ox = -1; ox <= 1; ++ox)", "for (int ox = -1; ox <= 0; ++ox)", 0,
                               [MD + "test_neighbour_list_cells_equal_brute_force"]),
    "stencil_y_wraps_by_nx": ("int32_t y = (cy + oy + nc[1]) % nc[1];", "int32_t y = (cy + oy + nc[1]) % nc[0];", 0,
                              [MD + "test_cells_and_lists_on_an_uneven_grid"]),
    "cell_decoded_with_nx_for_y": ("cy = (c / nc[0]) % nc[1]", "cy = (c / nc[0]) % nc[0]", 0,
                                   [MD + "test_cells_and_lists_on_an_uneven_grid"]),
    "cell_index_with_nx_twice": ("cell_of[i] = (cz * nc[1] + cy) * nc[0] + cx;",
                                 "cell_of[i] = (cz * nc[0] + cy) * nc[0] + cx;", 0,
                                 [MD + "test_cells_and_lists_on_an_uneven_grid"]),
    "cell_count_rounded": ("nc[d] = (int32_t)floor(L[d] / r);", "nc[d] = (int32_t)rint(L[d] / r);", 0,
                           [MD + "test_neighbour_list_cells_equal_brute_force"]),
    # Lennard-Jones pair loop, Eqs. (9) and (12)
    "force_sign_x": ("fx += fmag * dr[0];", "fx -= fmag * dr[0];", 0,
                     [MD + "test_force_is_minus_energy_gradient"]),
    "force_exponent_12": ("double sr14 = sr12 * sr2;", "double sr14 = sr12;", 0,
                          [MD + "test_force_is_minus_energy_gradient"]),
    "force_prefactor_24": ("double fmag = 48.0 * eps / s2", "double fmag = 24.0 * eps / s2", 0,
                           [MD + "test_force_is_minus_energy_gradient"]),
    "energy_not_halved": ("ei += 0.5 * 4.0 * eps", "ei += 4.0 * eps", 0,
                          [MD + "test_lattice_energy_closed_form"]),
    "sigma_left_out_of_the_ratio": ("double sr2 = s2 / r2;", "double sr2 = 1.0 / r2;", 0,
                                    [MD + "test_lj_scales_with_epsilon_and_sigma"]),
    "force_prefactor_without_sigma": ("double fmag = 48.0 * eps / s2", "double fmag = 48.0 * eps", 0,
                                      [MD + "test_lj_scales_with_epsilon_and_sigma"]),
    "energy_without_epsilon": ("ei += 0.5 * 4.0 * eps * (", "ei += 0.5 * 4.0 * (", 0,
                               [MD + "test_lj_scales_with_epsilon_and_sigma"]),
    "shift_sign": ("(sr12 - sr6 + shift)", "(sr12 - sr6 - shift)", 0,
                   [MD + "test_lattice_energy_closed_form"]),
    "virial_not_halved": ("wsum += 0.5 * fmag * r2;", "wsum += fmag * r2;", 0,
                          [MD + "test_virial_is_volume_derivative"]),
    # Velocity Verlet, Algorithm 6
    "kick_full_step": ("double h = dt / (2.0 * mass);", "double h = dt / mass;", 0,
                       [MD + "test_vv_constant_force_closed_form"]),
    "drift_half_step": ("pos[3 * i + d] + dt * vel[3 * i + d]", "pos[3 * i + d] + h * vel[3 * i + d]", 0,
                        [MD + "test_vv_constant_force_closed_form"]),
    "kinetic_not_halved": ("k += 0.5 * mass *", "k += mass *", 0,
                           [MD + "test_vv_energy_error_is_second_order"]),
    "list_never_rebuilt": ("if (rebuild_every > 0 && s % rebuild_every == 0) {",
                           "if (rebuild_every < 0 && s % rebuild_every == 0) {", 1,
                           [MD + "test_md_rebuild_policy_matches_fresh_lists"]),
    # bond order, Eqs. (4)-(5)
    "legendre_recurrence_index": ("- (ll + m - 1.0) * pmm) / (ll - m);", "- (ll + m) * pmm) / (ll - m);", 0,
                                  [AN + "test_perfect_lattice_Q_matches_paper_table"]),
    "ylm_norm_2pi": ("(2.0 * l + 1.0) / (4.0 * ORA_PI)", "(2.0 * l + 1.0) / (2.0 * ORA_PI)", 0,
                     [AN + "test_perfect_lattice_Q_matches_paper_table"]),
    "q_prefactor_2l": ("sqrt(4.0 * ORA_PI / (2.0 * l + 1.0) * s)", "sqrt(4.0 * ORA_PI / (2.0 * l) * s)", 0,
                       [AN + "test_perfect_lattice_Q_matches_paper_table"]),
    "bonnet_sign": ("(2.0 * k + 1.0) * x * p1 - k * p0", "(2.0 * k + 1.0) * x * p1 + k * p0", 0,
                    [AN + "test_Q_direct_equals_addition_theorem"]),
    "ylm_azimuth_without_m": ("yi = p * sin(am * phi);", "yi = p * sin(phi);", 0,
                              [AN + "test_Q_direct_equals_addition_theorem"]),
    # common neighbour analysis, Eqs. (6)-(8), Algorithms 3-5 and 7
    "cna_common_not_tested": ("if (in_set(&direct[eoff[j]], nu_nb[j], v)) C[nc++] = v;",
                              "if (v != j) C[nc++] = v;", 0,
                              [AN + "test_perfect_lattice_cna_signatures"]),
    "cna_bonds_not_deduplicated": ("if (!dup) {", "if (1) {", 0,
                                   [AN + "test_perfect_lattice_cna_signatures"]),
    "cluster_sum_not_max": ("if (S > smax) smax = S;", "smax += S;", 0,
                            [AN + "test_perfect_lattice_cna_signatures"]),
    "cluster_counts_first_edge_only": ("S += 1;", "S = 1;", 0,
                                       [AN + "test_perfect_lattice_cna_signatures"]),
    "label_hcp_as_bcc": ("c422 == 6) lab = 2;", "c422 == 6) lab = 3;", 0,
                         [AN + "test_perfect_lattice_cna_signatures"]),
    # features of the learned classifier
    "feature_distance_scale": ("(d[k] - r_ref) / (r_feat - r_ref)", "(d[k] - r_ref) / r_feat", 0,
                               [AN + "test_features_perfect_fcc_closed_form"]),
    "feature_tent_weights_swapped": ("f[16 + b0] += 1.0 - t;", "f[16 + b0] += t;", 0,
                                     [AN + "test_features_perfect_fcc_closed_form"]),
    "feature_histogram_norm": ("f[16 + b] /= 24.0;", "f[16 + b] /= 12.0;", 0,
                               [AN + "test_features_perfect_fcc_closed_form"]),
    # Philox4x32-10 and the Andersen thermostat (Sec. 5.2)
    "philox_multiplier": ("mulhilo32(0xCD9E8D57u, c2, &lo1)", "mulhilo32(0xCD9E8D59u, c2, &lo1)", 0,
                          [MD + "test_philox4x32_known_answers"]),
    "philox_weyl_constant": ("k1 += 0xBB67AE85u;", "k1 += 0x9E3779B9u;", 0,
                             [MD + "test_philox4x32_known_answers"]),
    "philox_nine_rounds": ("for (int r = 0; r < 10; ++r) {", "for (int r = 0; r < 9; ++r) {", 0,
                           [MD + "test_philox4x32_known_answers"]),
    "andersen_threshold_rounded_up": ("return (uint64_t)floor(p * 4294967296.0);",
                                      "return (uint64_t)ceil(p * 4294967296.0);", 0,
                                      [MD + "test_andersen_threshold"]),
    "box_muller_cos_twice": ("v[1] = sd * (r1 * sin(t1));", "v[1] = sd * (r1 * cos(t1));", 0,
                             [MD + "test_andersen_every_atom_every_step"]),
    # adaptive CNA (Stukowski 2012, cited in Sec. 4.2)
    "acna_factor": ("const double f = (1.0 + sqrt(2.0)) * 0.5;", "const double f = (1.0 + sqrt(3.0)) * 0.5;", 0,
                    [AN + "test_acna_perfect_lattices_at_any_density"]),
    "acna_bcc_weight_on_second_shell": ("rc14 = f * ((c * s8 + s6) / 14.0);", "rc14 = f * ((s8 + c * s6) / 14.0);",
                                        0, [AN + "test_acna_perfect_lattices_at_any_density"]),
    # more of the same regions, each with the pin that catches it
    "brute_force_lists_the_atom_itself": ("if (j == i) continue;", "if (0) continue;", 0,
                                          [MD + "test_neighbour_list_cells_equal_brute_force"]),
    "cell_prefix_sum_one_short": ("for (int64_t c = 0; c < ncell; ++c) cell_start[c + 1] += cell_start[c];",
                                  "for (int64_t c = 0; c + 1 < ncell; ++c) cell_start[c + 1] += cell_start[c];", 0,
                                  [MD + "test_lattice_energy_closed_form"]),
    "wrap_upper_edge_kept": ("if (y >= L) y = 0.0;", "if (y > L) y = 0.0;", 0,
                             [MD + "test_wrap_maps_into_the_half_open_box"]),
    "force_cutoff_ignored": ("            if (!(r2 < rc2)) continue;\n            double sr2", "            double sr2", 0,
                             [MD + "test_newton_third_law_and_energy_sum"]),
    "second_kick_also_drifts": ("if (phase == 1) pos[3 * i + d]", "if (phase >= 1) pos[3 * i + d]", 0,
                                [MD + "test_vv_constant_force_closed_form"]),
    "potential_energy_halved": ("energies[2 * (s - 1) + 1] = U;", "energies[2 * (s - 1) + 1] = 0.5 * U;", 1,
                                [MD + "test_vv_energy_error_is_second_order"]),
    "skin_guard_not_a_maximum": ("if (d2 > md2) md2 = d2;", "md2 = d2;", 1,
                                 [MD + "test_md_max_displacement_since_rebuild"]),
    "skin_guard_reference_kept": ("memcpy(ref, pos, sizeof(double) * (size_t)(3 * n));\n        }", "}", 1,
                                  [MD + "test_md_max_displacement_since_rebuild"]),
    "ylm_factorials_swapped": ("factorial(l - am) / factorial(l + am)", "factorial(l + am) / factorial(l - am)", 0,
                               [MD + "test_otf_q_rows_of_a_crystal_at_rest"]),
    "q_rows_mean_over_n_minus_1": ("sum / (double)(n > 0 ? n : 1)", "sum / (double)(n > 1 ? n - 1 : 1)", 0,
                                   [MD + "test_otf_q_rows_of_a_crystal_at_rest"]),
    "q_rows_one_step_early": ("if (boa_every > 0 && s % boa_every == 0) {",
                              "if (boa_every > 0 && (s - 1) % boa_every == 0) {", 0,
                              [MD + "test_otf_q_rows_of_a_crystal_at_rest"]),
    "andersen_second_draw_counter": ("ctr[3] = 1u;", "ctr[3] = 2u;", 0, [MD + "test_andersen_every_atom_every_step"]),
    "andersen_counter_words_swapped": ("uint32_t ctr[4] = {(uint32_t)id, (uint32_t)step,",
                                       "uint32_t ctr[4] = {(uint32_t)step, (uint32_t)id,", 0,
                                       [MD + "test_andersen_every_atom_every_step"]),
    "cna_bonds_capped_at_12": ("nbond[i] = ni;", "nbond[i] = ni < 12 ? ni : 12;", 0,
                               [AN + "test_perfect_lattice_cna_signatures"]),
    "bcc_signature_counts_swapped": ("nb == 14 && c666 == 8 && c444 == 6) lab = 3;",
                                     "nb == 14 && c666 == 6 && c444 == 8) lab = 3;", 0,
                                     [AN + "test_perfect_lattice_cna_signatures"]),
    "feature_q_at_the_bond_length": ("ora_boa_direct(n, pos, L, r_feat, offs, nbr, 4, q4, NULL);",
                                     "ora_boa_direct(n, pos, L, r_ref, offs, nbr, 4, q4, NULL);", 0,
                                     [AN + "test_features_shell_between_the_cutoffs"]),
    "feature_bonds_at_the_feature_cutoff": ("if (!(r2 < r_ref * r_ref)) continue;", "if (!(r2 < rc2)) continue;", 0,
                                            [AN + "test_features_shell_between_the_cutoffs"]),
    "feature_distances_unsorted": ("qsort(d, (size_t)nu, sizeof(double), cmp_f64);", ";", 0,
                                   [AN + "test_features_rotation_invariant_and_counts"]),
    "feature_missing_distance_zero": ("(k < nu) ? (d[k] - r_ref) / (r_feat - r_ref) : 1.0;",
                                      "(k < nu) ? (d[k] - r_ref) / (r_feat - r_ref) : 0.0;", 0,
                                      [AN + "test_features_perfect_fcc_closed_form"]),
    "acna_skips_the_nearest": ("for (int a = 0; a < 12; ++a) {\n                s += sqrt(cand[a].r2);",
                               "for (int a = 1; a < 13; ++a) {\n                s += sqrt(cand[a].r2);", 0,
                               [AN + "test_acna_perfect_lattices_at_any_density"]),
    "addition_route_self_pairs_dropped": ("for (int b = 0; b < nu; ++b) {\n                double c = u[3 * a]",
                                          "for (int b = 0; b < nu; ++b) if (b != a) {\n                double c = u[3 * a]",
                                          0, [AN + "test_Q_direct_equals_addition_theorem"]),
    "addition_route_divides_by_nu_squared": ("Q[i] = sqrt(s) / nu;", "Q[i] = sqrt(s) / ((double)nu * nu);", 0,
                                             [AN + "test_Q_direct_equals_addition_theorem"]),
    "q5_skipped_in_the_run": ("for (int l = 4; l <= 6; ++l) {", "for (int l = 4; l <= 6; l += 1 + (l == 4)) {", 0,
                              [MD + "test_otf_q_rows_of_hcp_at_rest"]),
    "stencil_wraps_by_n_plus_1": ("int32_t x = (cx + ox + nc[0]) % nc[0];", "int32_t x = (cx + ox + nc[0]) % (nc[0] + 1);",
                                  0, [MD + "test_lattice_energy_closed_form"]),
    "energy_attractive_term_sign": ("ei += 0.5 * 4.0 * eps * (sr12 - sr6 + shift);",
                                    "ei += 0.5 * 4.0 * eps * (sr12 + sr6 + shift);", 0,
                                    [MD + "test_lattice_energy_closed_form"]),
    "kinetic_without_mass": ("k += 0.5 * mass *", "k += 0.5 *", 0, [MD + "test_vv_energy_error_is_second_order"]),
    "rebuild_at_the_force_cutoff": ("build_list_cells(n, pos, L, r_list, offs, &nbr, &cap);\n            memcpy",
                                    "build_list_cells(n, pos, L, rc, offs, &nbr, &cap);\n            memcpy", 1,
                                    [MD + "test_md_rebuild_policy_matches_fresh_lists"]),
    "philox_output_words_swapped": ("out[1] = c1;\n    out[2] = c2;", "out[1] = c2;\n    out[2] = c1;", 0,
                                    [MD + "test_philox4x32_known_answers"]),
    "philox_low_and_high_halves": ("c1 = lo1;", "c1 = hi1;", 0, [MD + "test_philox4x32_known_answers"]),
    "thermostat_before_the_second_kick": (
        "ora_vv(2, n, pos, vel, F, L, mass, dt);\n        if (energies) {\n            energies[2 * (s - 1)] = "
        "ora_kinetic(n, vel, mass);\n            energies[2 * (s - 1) + 1] = U;\n        }\n        if (thr > 0)\n"
        "            for (int64_t i = 0; i < n; ++i) ncoll += andersen_draw(seed, i, s, thr, sd, &vel[3 * i]);",
        "if (thr > 0)\n            for (int64_t i = 0; i < n; ++i) ncoll += andersen_draw(seed, i, s, thr, sd, "
        "&vel[3 * i]);\n        ora_vv(2, n, pos, vel, F, L, mass, dt);\n        if (energies) {\n            "
        "energies[2 * (s - 1)] = ora_kinetic(n, vel, mass);\n            energies[2 * (s - 1) + 1] = U;\n        }",
        0, [MD + "test_andersen_every_atom_every_step"]),
    "andersen_spread_without_mass": ("const double sd = sqrt(T / mass);", "const double sd = sqrt(T);", 0,
                                     [MD + "test_andersen_draws_have_variance_t_over_m"]),
    "box_muller_radius_not_rooted": ("const double r1 = sqrt(-2.0 * log(U1)), t1 = two_pi * U2;",
                                     "const double r1 = -2.0 * log(U1), t1 = two_pi * U2;", 0,
                                     [MD + "test_andersen_every_atom_every_step"]),
    "uniform_without_the_half": ("const double U1 = ((double)u[1] + 0.5) * inv32", "const double U1 = ((double)u[1]) * inv32",
                                 0, [MD + "test_andersen_every_atom_every_step"]),
    "cluster_neighbour_not_queued": ("if (!seen) Q[qn++] = w;", "if (0) Q[qn++] = w;", 0,
                                     [AN + "test_perfect_lattice_cna_signatures"]),
    "acna_triplet_counts_the_bond_partner": (
        "if (b != a && min_image(&pos[3 * sel[a]], &pos[3 * sel[b]], L, dr) < rc2) cn[ncn++] = sel[b];",
        "if (min_image(&pos[3 * sel[a]], &pos[3 * sel[b]], L, dr) < rc2) cn[ncn++] = sel[b];", 0,
        [AN + "test_acna_perfect_lattices_at_any_density"]),
    "acna_bcc_test_overrides_fcc": ("if (lab == 0 && deg >= 14) {", "if (deg >= 14) {", 0,
                                    [AN + "test_acna_perfect_lattices_at_any_density"]),
    "chord_from_the_sum_of_bonds": (
        "double cx = u[3 * a] - u[3 * b], cy = u[3 * a + 1] - u[3 * b + 1], cz = u[3 * a + 2] - u[3 * b + 2];",
        "double cx = u[3 * a] + u[3 * b], cy = u[3 * a + 1] + u[3 * b + 1], cz = u[3 * a + 2] + u[3 * b + 2];", 0,
        [AN + "test_features_perfect_fcc_closed_form"]),
    "histogram_low_edge_shifted": ("double lo = r_ref - 0.35;", "double lo = r_ref - 0.30;", 0,
                                   [AN + "test_features_perfect_fcc_closed_form"]),
    "fcc_label_with_10_of_12": ("if (nb == 12 && c421 == 12) lab = 1;", "if (nb == 12 && c421 >= 10) lab = 1;", 0,
                                [AN + "test_cna_label_rule_needs_the_exact_signature"]),
    "hcp_label_from_any_mix": ("else if (nb == 12 && c421 == 6 && c422 == 6) lab = 2;",
                               "else if (nb == 12 && c421 + c422 == 12) lab = 2;", 0,
                               [AN + "test_cna_label_rule_needs_the_exact_signature"]),
    "bcc_label_loosened": ("else if (nb == 14 && c666 == 8 && c444 == 6) lab = 3;",
                           "else if (nb >= 13 && c666 >= 7 && c444 >= 6) lab = 3;", 0,
                           [AN + "test_cna_label_rule_needs_the_exact_signature"]),
    "rebuild_one_step_early": ("if (rebuild_every > 0 && s % rebuild_every == 0) {",
                               "if (rebuild_every > 0 && (s + 1) % rebuild_every == 0) {", 1,
                               [MD + "test_md_max_displacement_since_rebuild"]),
    "q_of_a_lone_atom_one": ("        if (nu == 0) {\n            Q[i] = 0.0;\n            continue;\n        }\n"
                             "        double s = 0.0;\n        for (int m",
                             "        if (nu == 0) {\n            Q[i] = 1.0;\n            continue;\n        }\n"
                             "        double s = 0.0;\n        for (int m", 0,
                             [AN + "test_bond_order_of_an_atom_without_bonds_is_zero"]),
    "cells_of_unwrapped_coordinates": ("double xw = wrap1(x, L);", "double xw = x;", 0,
                                       [MD + "test_cells_and_lists_on_an_uneven_grid"]),
    "min_image_y_counted_twice": ("return dr[0] * dr[0] + dr[1] * dr[1] + dr[2] * dr[2];",
                                  "return dr[0] * dr[0] + dr[1] * dr[1] + dr[1] * dr[1];", 0,
                                  [MD + "test_lattice_energy_closed_form"]),
    "kinetic_y_counted_twice": ("vel[3 * i + 2] * vel[3 * i + 2]);", "vel[3 * i + 1] * vel[3 * i + 1]);", 0,
                                [MD + "test_vv_energy_error_is_second_order"]),
    "histogram_centres_unshifted": ("double x = (chord - lo) / 0.05 - 0.5;", "double x = (chord - lo) / 0.05;", 0,
                                    [AN + "test_features_perfect_fcc_closed_form"]),
    "acna_bcc_scale_inverted": ("const double c = 2.0 / sqrt(3.0);", "const double c = sqrt(3.0) / 2.0;", 0,
                                [AN + "test_acna_perfect_lattices_at_any_density"]),
    "thirteen_distance_features": ("for (int k = 0; k < 14; ++k) f[2 + k] =", "for (int k = 0; k < 13; ++k) f[2 + k] =", 0,
                                   [AN + "test_features_perfect_fcc_closed_form"]),
}

# the classifier's network, forward and backward passes, AdamW (oracle/mlp.py)
MLP_MUTANTS = {
    "relu_mask_of_the_wrong_layer": ('d2 = (g3 @ p["W3"].T) * (z2 > 0)', 'd2 = (g3 @ p["W3"].T) * (z1 > 0)', 0,
                                     [AN + "test_mlp_gradient_matches_finite_differences"]),
    "backprop_weight_not_transposed": ('d1 = (d2 @ p["W2"].T)', 'd1 = (d2 @ p["W2"])', 0,
                                       [AN + "test_mlp_gradient_matches_finite_differences"]),
    "softmax_gradient_onehot_added": ("g3[np.arange(n), y] -= 1.0", "g3[np.arange(n), y] += 1.0", 0,
                                      [AN + "test_mlp_gradient_matches_finite_differences"]),
    "gradient_not_averaged": ("g3 /= n", "g3 /= 1", 0, [AN + "test_mlp_gradient_matches_finite_differences"]),
    "second_relu_dropped": ("h2 = np.maximum(z2, 0.0)", "h2 = z2", 0,
                            [AN + "test_mlp_gradient_matches_finite_differences"]),
    "standardisation_by_variance": ("1.0 / np.sqrt(np.maximum(var, 1e-300))", "1.0 / np.maximum(var, 1e-300)", 0,
                                    [AN + "test_mlp_input_standardisation"]),
    "adamw_no_bias_correction": ("mh = m / (1.0 - b1 ** t)", "mh = m", 0, [AN + "test_adamw_textbook_steps"]),
    "adamw_eps_inside_sqrt": ("np.sqrt(vh) + eps", "np.sqrt(vh + eps)", 0, [AN + "test_adamw_textbook_steps"]),
    "adamw_decay_not_decoupled": ("p[k] = p[k] - lr * wd * p[k]", "g = g + wd * p[k]", 0,
                                  [AN + "test_adamw_textbook_steps"]),
    "bf16_ties_away_from_even": ("r = ((u + 0x7FFF + keep_lsb) >> 16) << 16", "r = ((u + 0x8000) >> 16) << 16", 0,
                                 [BF + "test_bf16_round_matches_torch"]),
    "bf16_hidden_layer_unrounded": ("h1 = bf16_round(np.maximum(z1, 0.0))", "h1 = np.maximum(z1, 0.0)", 0,
                                    [BF + "test_forward_bf16_operands_are_bf16_values"]),
    "bf16_standardisation_reordered": ('(f32(x) - f32(p["mu"])) * f32(p["isd"])',
                                       'f32(x) * f32(p["isd"]) - f32(p["mu"])', 0,
                                       [BF + "test_forward_bf16_is_the_network_on_exact_operands",
                                        BF + "test_forward_bf16_differs_by_rounding_only"]),
    "loss_summed_not_averaged": ("loss = -np.mean(np.log(prob[np.arange(n), y]))",
                                 "loss = -np.sum(np.log(prob[np.arange(n), y]))", 0,
                                 [AN + "test_mlp_gradient_matches_finite_differences"]),
    "adamw_second_moment_unsquared": ("(1.0 - b2) * g * g", "(1.0 - b2) * g", 0, [AN + "test_adamw_textbook_steps"]),
    "constant_feature_scaled_to_zero": ("1.0 / np.sqrt(np.maximum(var, 1e-300)), 1.0)",
                                        "1.0 / np.sqrt(np.maximum(var, 1e-300)), 0.0)", 0,
                                        [AN + "test_mlp_input_standardisation"]),
    "bf16_bias_rounded": ('z1 = xs @ W1 + f32(p["b1"]).astype(np.float64)', 'z1 = xs @ W1 + bf16_round(p["b1"])', 0,
                          [BF + "test_tolerance_covers_fp32_accumulation"]),
    "bf16_last_weights_unrounded": ('W1, W2, W3 = (bf16_round(p[k]) for k in ("W1", "W2", "W3"))',
                                    'W1, W2, W3 = bf16_round(p["W1"]), bf16_round(p["W2"]), p["W3"]', 0,
                                    [BF + "test_forward_bf16_weights_enter_as_bf16"]),
    "softmax_shifted_by_the_minimum": ("z = logits - logits.max(axis=1, keepdims=True)",
                                       "z = logits - logits.min(axis=1, keepdims=True)", 0,
                                       [AN + "test_softmax_of_large_logits"]),
    "adamw_decay_without_lr": ("p[k] = p[k] - lr * wd * p[k]", "p[k] = p[k] - wd * p[k]", 0,
                               [AN + "test_adamw_textbook_steps"]),
    "adamw_second_moment_corrected_by_b1": ("vh = v / (1.0 - b2 ** t)", "vh = v / (1.0 - b1 ** t)", 0,
                                            [AN + "test_adamw_textbook_steps"]),
    "bias_gradient_from_the_wrong_layer": ('grads["b2"] = d2.sum(0)', 'grads["b2"] = d1.sum(0)', 0,
                                           [AN + "test_mlp_gradient_matches_finite_differences"]),
    "bf16_round_truncates": ("r = ((u + 0x7FFF + keep_lsb) >> 16) << 16", "r = (u >> 16) << 16", 0,
                             [BF + "test_bf16_round_matches_torch"]),
    "adamw_trains_the_scales": ('        if k in ("mu", "isd"):\n            continue  # fitted, not trained',
                                '        if k in ("mu",):\n            continue  # fitted, not trained', 0,
                                [AN + "test_mlp_input_standardisation"]),
    "bf16_standardised_inputs_unrounded": ('xs = bf16_round((f32(x) - f32(p["mu"])) * f32(p["isd"]))',
                                           'xs = (f32(x) - f32(p["mu"])) * f32(p["isd"])', 0,
                                           [BF + "test_forward_bf16_operands_are_bf16_values"]),
}

# the Python side of the oracle package (oracle/__init__.py): the bond-order
# tolerance rule of Sec. 4.1 and its table
PKG_MUTANTS = {
    "tolerance_edge_inclusive": ("np.where(best < tol, lab, np.int8(0))", "np.where(best <= tol, lab, np.int8(0))",
                                 0, [AN + "test_boa_tolerance_rule_edges"]),
    "tolerance_tie_to_the_later_lattice": ("closer = d < best", "closer = d <= best", 0,
                                           [AN + "test_boa_tolerance_rule_edges"]),
    "tolerance_table_hcp_q6": ("(2, 0.097, 0.485)", "(2, 0.097, 0.511)", 0,
                               [AN + "test_boa_tolerance_table_is_the_papers"]),
    "tolerance_distance_squared": ("d = np.sqrt((q4 - r4) ** 2 + (q6 - r6) ** 2)", "d = (q4 - r4) ** 2 + (q6 - r6) ** 2",
                                   0, [AN + "test_boa_tolerance_labels_perfect_lattices"]),
}

# the classifier parity tests' comparison helpers (tests/oracle_pipeline.py):
# the logit tolerance of a row and the labels admissible within it
PIPE_SRC = os.path.join(ROOT, "tests", "oracle_pipeline.py")
OP = "tests/test_oracle_pipeline_cpu.py::"
PIPE_MUTANTS = {
    "input_step_budget_x10": ("        tol *= 2.0", "        tol *= 20.0", 0,
                              [BF + "test_tolerance_covers_one_feature_step"]),
    "hidden_layer_step_dropped": ("    tol += (bf16_step(h1)[:, :, None] * np.abs(K1)).max(axis=(1, 2))\n", "", 0,
                                  [BF + "test_tolerance_covers_fp32_accumulation"]),
    "bf16_step_four_times_too_large": ("return np.where(a > 0, 2.0 ** (e - 7), 0.0)",
                                       "return np.where(a > 0, 2.0 ** (e - 5), 0.0)", 0,
                                       [BF + "test_tolerance_covers_one_feature_step"]),
    "leading_window_x10": ("cand = logits >= (top - 2.0 * tol)[:, None]", "cand = logits >= (top - 20.0 * tol)[:, None]",
                           0, [OP + "test_hand_worked_rows"]),
    "probability_move_x10": ("dp = 3.0 * pmax * (1.0 - pmax) * tol + 1e-6", "dp = 30.0 * pmax * (1.0 - pmax) * tol + 1e-6",
                             0, [OP + "test_hand_worked_rows"]),
    "cna_label_always_admissible": ("can_fall = pmax - dp < threshold", "can_fall = pmax - dp < 2.0", 0,
                                    [OP + "test_no_tolerance_admits_the_rule_alone"]),
    "every_class_admissible": ("ok[can_keep] = cand[can_keep]", "ok[can_keep] = True", 0,
                               [OP + "test_no_tolerance_admits_the_rule_alone"]),
}

# the child process for a Python mutant: the copy is imported under the
# module's own name before pytest imports any test module.  `path` is
# oracle/mlp.py's copy, tests/oracle_pipeline.py's (saved under that file
# name), or the directory holding a copy of the package.
_PY_BOOT = """import importlib.util, os, sys
sys.path.insert(0, {root!r})
path = {path!r}
if os.path.isdir(path):
    sys.path.insert(0, path)
    import oracle
    assert os.path.dirname(oracle.__file__) == os.path.join(path, "oracle")
elif path.endswith("oracle_pipeline.py"):
    sys.path.insert(0, os.path.join({root!r}, "tests"))
    spec = importlib.util.spec_from_file_location("oracle_pipeline", path)
    m = importlib.util.module_from_spec(spec)
    sys.modules["oracle_pipeline"] = m
    spec.loader.exec_module(m)
else:
    import oracle
    spec = importlib.util.spec_from_file_location("oracle.mlp", path)
    m = importlib.util.module_from_spec(spec)
    sys.modules["oracle.mlp"] = m
    spec.loader.exec_module(m)
    oracle.mlp = m
import pytest
sys.exit(pytest.main({args!r}))
"""


def plant(src, old, new, occurrence):
    """The source with the given occurrence of `old` replaced by `new`."""
    at = -1
    for _ in range(occurrence + 1):
        at = src.find(old, at + 1)
        assert at >= 0, f"{old!r}: occurrence {occurrence} not in the oracle's source"
    return src[:at] + new + src[at + len(old):]


def run_pins(pins, lib=None, py=None):
    """Run the pins against the oracle build `lib`, or the Python copy `py`
    (see _PY_BOOT; None: the repository's own); (pytest's exit code, the
    tail of its output)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    if lib:
        env["PPMD_ORACLE_LIB"] = lib
    args = ["-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu", *pins]
    if py:
        cmd = [sys.executable, "-c", _PY_BOOT.format(root=ROOT, path=py, args=args)]
    else:
        cmd = [sys.executable, "-m", "pytest", *args]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr)[-1500:]


def _mutant(kind, name, tmp):
    import oracle
    if kind == "c":
        old, new, occurrence, pins = MUTANTS[name]
        src = os.path.join(tmp, f"{name}.c")
        with open(SRC) as f, open(src, "w") as g:
            g.write(plant(f.read(), old, new, occurrence))
        lib = os.path.join(tmp, f"{name}.so")
        oracle.compile_source(src, lib)
        return run_pins(pins, lib=lib)
    if kind == "py":
        old, new, occurrence, pins = MLP_MUTANTS[name]
        path = os.path.join(tmp, f"{name}.py")
        with open(MLP_SRC) as f, open(path, "w") as g:
            g.write(plant(f.read(), old, new, occurrence))
        return run_pins(pins, py=path)
    if kind == "pipe":
        old, new, occurrence, pins = PIPE_MUTANTS[name]
        os.makedirs(os.path.join(tmp, name))
        path = os.path.join(tmp, name, "oracle_pipeline.py")
        with open(PIPE_SRC) as f, open(path, "w") as g:
            g.write(plant(f.read(), old, new, occurrence))
        return run_pins(pins, py=path)
    old, new, occurrence, pins = PKG_MUTANTS[name]
    top = copy_package(os.path.join(tmp, name))
    init = os.path.join(top, "oracle", "__init__.py")
    with open(init) as f:
        src = plant(f.read(), old, new, occurrence)
    with open(init, "w") as g:
        g.write(src)
    return run_pins(pins, py=top)


def copy_package(top):
    """A copy of the oracle package's sources under top/oracle; returns top."""
    os.makedirs(os.path.join(top, "oracle"))
    for f in os.listdir(os.path.dirname(SRC)):
        if f.endswith((".py", ".c")):
            shutil.copy(os.path.join(os.path.dirname(SRC), f), os.path.join(top, "oracle", f))
    return top


@pytest.fixture(scope="module")
def results():
    """Every mutant made and its pins run, several at a time."""
    with tempfile.TemporaryDirectory() as tmp:
        with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
            futs = {("c", k): ex.submit(_mutant, "c", k, tmp) for k in MUTANTS}
            futs.update({("py", k): ex.submit(_mutant, "py", k, tmp) for k in MLP_MUTANTS})
            futs.update({("pkg", k): ex.submit(_mutant, "pkg", k, tmp) for k in PKG_MUTANTS})
            futs.update({("pipe", k): ex.submit(_mutant, "pipe", k, tmp) for k in PIPE_MUTANTS})
            yield {key: f.result() for key, f in futs.items()}


@pytest.mark.parametrize("table,path", [(MUTANTS, SRC), (MLP_MUTANTS, MLP_SRC), (PKG_MUTANTS, PKG_SRC),
                                        (PIPE_MUTANTS, PIPE_SRC)], ids=["c", "mlp", "package", "pipeline"])
def test_every_mistake_is_planted_where_named(table, path):
    """Each mistake changes the source at the named place."""
    with open(path) as f:
        src = f.read()
    for name, (old, new, occurrence, pins) in table.items():
        assert old != new and pins, name
        assert src.count(old) >= occurrence + 1, name
        assert plant(src, old, new, occurrence) != src, name


def test_unchanged_sources_pass_the_pins():
    """The same four routes with nothing planted: the pins pass on a fresh
    build of the oracle's own C source, on copies of its network and of the
    package, and on a copy of the comparison helpers."""
    import oracle
    c_pins = sorted({p for *_, ps in MUTANTS.values() for p in ps})
    py_pins = sorted({p for *_, ps in MLP_MUTANTS.values() for p in ps})
    pkg_pins = sorted({p for *_, ps in PKG_MUTANTS.values() for p in ps})
    pipe_pins = sorted({p for *_, ps in PIPE_MUTANTS.values() for p in ps})
    with tempfile.TemporaryDirectory() as tmp:
        lib = os.path.join(tmp, "unchanged.so")
        oracle.compile_source(SRC, lib)
        code, out = run_pins(c_pins, lib=lib)
        assert code == 0, out
        path = os.path.join(tmp, "unchanged_mlp.py")
        with open(MLP_SRC) as f, open(path, "w") as g:
            g.write(f.read())
        code, out = run_pins(py_pins, py=path)
        assert code == 0, out
        code, out = run_pins(pkg_pins, py=copy_package(os.path.join(tmp, "unchanged_package")))
        assert code == 0, out
        os.makedirs(os.path.join(tmp, "unchanged_pipeline"))
        path = os.path.join(tmp, "unchanged_pipeline", "oracle_pipeline.py")
        with open(PIPE_SRC) as f, open(path, "w") as g:
            g.write(f.read())
        code, out = run_pins(pipe_pins, py=path)
        assert code == 0, out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_the_mistake(results, name):
    code, out = results[("c", name)]
    assert code == 1, f"{name}: the pins {MUTANTS[name][3]} did not fail (pytest exit {code}):\n{out}"


@pytest.mark.parametrize("name", sorted(MLP_MUTANTS))
def test_pins_catch_the_network_mistake(results, name):
    code, out = results[("py", name)]
    assert code == 1, f"{name}: the pins {MLP_MUTANTS[name][3]} did not fail (pytest exit {code}):\n{out}"


@pytest.mark.parametrize("name", sorted(PKG_MUTANTS))
def test_pins_catch_the_package_mistake(results, name):
    code, out = results[("pkg", name)]
    assert code == 1, f"{name}: the pins {PKG_MUTANTS[name][3]} did not fail (pytest exit {code}):\n{out}"


@pytest.mark.parametrize("name", sorted(PIPE_MUTANTS))
def test_pins_catch_the_comparison_mistake(results, name):
    code, out = results[("pipe", name)]
    assert code == 1, f"{name}: the pins {PIPE_MUTANTS[name][3]} did not fail (pytest exit {code}):\n{out}"
