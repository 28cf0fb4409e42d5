"""Mutation check of the oracle's pins.

Every GPU parity test compares the CUDA path with the oracle, so a mistake in
the oracle that its own pins let through would pass unnoticed everywhere.
Each case below plants one plausible mistake in a copy of the oracle's C
source -- a dropped term or factor, a flipped sign, a wrong index or
constant, swapped operands, a step taken at the wrong point of the stage --
builds that copy, routes the oracle's Python wrappers through it and runs the
pins that should notice.  At least one of them must fail with an assertion
(any other exception is a fault of the harness, not a detection).

The planted edits are exact source substrings: a case whose text no longer
occurs in the oracle fails loudly, so the list follows the oracle's changes.
"""
import ctypes as C
import inspect
import itertools
import os
import tempfile
import textwrap
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import test_oracle_pins as P
import test_oracle_pins_adapt as A

# (name, edits, pins).  An edit is (old, new) -- old must occur exactly once --
# or (old, new, count) for a mistake repeated at `count` places.
MUTANTS = [
    # Philox4x32-10 (published definition; known answers)
    ("philox_weyl_constant", [("k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;")],
     [P.test_philox_known_answers]),
    ("philox_output_words_swapped", [("c1 = lo1;", "c1 = lo0;"), ("c3 = lo0;", "c3 = lo1;")],
     [P.test_philox_known_answers]),
    ("uniform_closed_at_zero", [("return ((double)k + 0.5) * 2.3283064365386963e-10;",
                                 "return ((double)k) * 2.3283064365386963e-10;")],
     [P.test_uniform_mapping_is_open_interval]),
    ("box_muller_radius", [("sqrt(-2.0 * log(u01(a)))", "sqrt(-log(u01(a)))")],
     [P.test_prior_draw_distributions]),
    # peak profiles (Eq. (C1), Eq. (E1))
    ("pv_mixing_swapped", [("return A * (eta * gau + (1.0 - eta) * lor);",
                            "return A * ((1.0 - eta) * gau + eta * lor);")],
     [P.test_peak_areas]),
    ("pv_gauss_part_hwhm_as_sd", [("double s = w / sqrt(2.0 * log(2.0));", "double s = w;")],
     [P.test_pv_height_and_half_height]),
    ("lorentz_width_not_squared", [("double lor = w * w / (w * w + dx * dx);",
                                    "double lor = w / (w + dx * dx);")],
     [P.test_gauss_lorentz_half_heights]),
    ("gauss_sd_missing_two", [("return A * exp(-dx * dx / (2.0 * w * w));",
                               "return A * exp(-dx * dx / (w * w));")],
     [P.test_gauss_lorentz_half_heights]),
    ("gauss_precision_missing_half", [("return A * exp(-w * dx * dx / 2.0);",
                                       "return A * exp(-w * dx * dx);")],
     [P.test_precision_gaussian_height_half_height_area]),
    # Chebyshev background (Eq. (1))
    ("chebyshev_recurrence_sign", [("double c = 2.0 * t * b - a;", "double c = 2.0 * t * b + a;")],
     [P.test_background_is_chebyshev_series]),
    ("chebyshev_grid_map", [("double t = (2.0 * x - (xmin + xmax)) / (xmax - xmin);",
                             "double t = (x - xmin) / (xmax - xmin);")],
     [P.test_background_is_chebyshev_series]),
    ("background_coefficient_index", [("f += nat[p * K + j] * chebyshev(j, t);",
                                       "f += nat[p * K] * chebyshev(j, t);")],
     [P.test_background_is_chebyshev_series]),
    # energies and likelihood normalisers (Eq. (C2), App. E, Eq. (D8))
    ("energy_half_dropped", [("e += 0.5 * r * r;", "e += r * r;", 2)],
     [P.test_energy_brute_force_high_precision, P.test_evidence_linear_gaussian_closed_form]),
    ("sigma_dropped_in_run_energy", [(" /\n                   job->sigma[i];", ";")],
     [P.test_evidence_linear_gaussian_closed_form, P.test_evidence_k1_quadrature_gamma_amplitude,
      P.test_evidence_k1_quadrature_free_centre]),
    ("gaussian_normaliser_missing_sqrt_2pi", [("lognorm -= log(sqrt(2.0 * M_PI) * job->sigma[i]);",
                                               "lognorm -= log(job->sigma[i]);")],
     [P.test_evidence_linear_gaussian_closed_form, P.test_evidence_k1_quadrature_gamma_amplitude]),
    ("model_variance_log_term_dropped", [("e += 0.5 * log(2.0 * M_PI * v) + 0.5 * r * r / v;",
                                          "e += 0.5 * r * r / v;", 2)],
     [P.test_energy_model_variance_brute_force, P.test_evidence_k1_quadrature_model_variance_shirley]),
    ("model_variance_linear_coefficient", [
        ("double v = s0 * s0 * f[i] + s1 * s1 * f[i] * f[i] + s2 * s2;",
         "double v = s0 * f[i] + s1 * s1 * f[i] * f[i] + s2 * s2;"),
        ("double v = np_[0] * np_[0] * f[i] + np_[1] * np_[1] * f[i] * f[i] + np_[2] * np_[2];",
         "double v = np_[0] * f[i] + np_[1] * np_[1] * f[i] * f[i] + np_[2] * np_[2];")],
     [P.test_energy_model_variance_brute_force, P.test_evidence_k1_quadrature_model_variance_shirley]),
    ("shirley_direction_reversed", [("double shirley = total > 0.0 ? a + (b - a) * run / total : a;",
                                     "double shirley = total > 0.0 ? b + (a - b) * run / total : a;")],
     [P.test_shirley_background_endpoints_and_gaussian_closed_form]),
    ("shirley_left_rectangle", [("if (i > 0) run += f[i] * fabs(x[i] - x[i - 1]);",
                                 "if (i > 0) run += f[i - 1] * fabs(x[i] - x[i - 1]);")],
     [P.test_shirley_background_endpoints_and_gaussian_closed_form]),
    ("poisson_log_term_sign", [("return (f - y) - y * log(f / y);", "return (f - y) + y * log(f / y);")],
     [P.test_xrd_poisson_log_z_of_fixed_background_is_exact, P.test_xrd_evidence_k1_quadrature_amplitude]),
    ("poisson_zero_count_term", [("if (y == 0.0) return f;", "if (y == 0.0) return 0.0;")],
     [P.test_xrd_poisson_zero_counts]),
    ("poisson_normaliser_missing_lgamma", [
        ("lognorm += (y > 0.0 ? y * log(y) : 0.0) - y - lgamma(y + 1.0);",
         "lognorm += (y > 0.0 ? y * log(y) : 0.0) - y;")],
     [P.test_xrd_poisson_log_z_of_fixed_background_is_exact]),
    # XRD phase model (App. D)
    ("caglioti_v_sign", [("double rad = u * tn * tn - v * tn + w;", "double rad = u * tn * tn + v * tn + w;")],
     [P.test_xrd_widths_at_ninety_degrees, P.test_xrd_phase_model_matches_independent_synthesis]),
    ("half_angle_not_halved", [("double th = x * M_PI / 360.0;", "double th = x * M_PI / 180.0;")],
     [P.test_xrd_widths_at_ninety_degrees, P.test_xrd_phase_model_matches_independent_synthesis]),
    ("asymmetry_on_wrong_side", [("asym = x >= mu ? alpha : 1.0;", "asym = x >= mu ? 1.0 : alpha;")],
     [P.test_xrd_phase_model_matches_independent_synthesis]),
    ("zero_shift_sign", [("double mu = pos[j] + shift,", "double mu = pos[j] - shift,")],
     [P.test_xrd_phase_model_matches_independent_synthesis]),
    ("xrd_pv_mixing_swapped", [("return (1.0 - r) * g + r * l;", "return r * g + (1.0 - r) * l;")],
     [P.test_xrd_phase_reduces_to_gaussian_peak, P.test_xrd_phase_model_matches_independent_synthesis]),
    ("xrd_background_offset_dropped", [("return bg[0] * xrd_pv(x, bg[1], bg[1], bg[2]) + bg[3]; }",
                                        "return bg[0] * xrd_pv(x, bg[1], bg[1], bg[2]); }")],
     [P.test_xrd_background_closed_form]),
    # prior draws and prior densities (Sec. II B 2)
    ("gamma_small_shape_not_boosted", [("double a = pr.p1 < 1.0 ? pr.p1 + 1.0 : pr.p1;", "double a = pr.p1;")],
     [P.test_prior_draw_distributions]),
    ("chebyshev_second_kind", [("double a = 1.0, b = t;", "double a = 1.0, b = 2.0 * t;")],
     [P.test_background_is_chebyshev_series]),
    ("mh_normal_from_one_word", [("box_muller(ww[0], ww[1])", "box_muller(ww[0], ww[0])")],
     [P.test_mh_keeps_prior_at_beta_zero, P.test_mh_keeps_gaussian_posterior_invariant]),
    ("mh_accept_uniform_from_a_normal_word", [("log(u01(ww[2]))", "log(u01(ww[0]))")],
     [P.test_mh_keeps_gaussian_posterior_invariant, P.test_mh_keeps_prior_at_beta_zero]),
    ("gamma_rate_read_as_scale", [("return g / pr.p2;", "return g * pr.p2;")],
     [P.test_prior_draw_distributions]),
    ("gamma_small_shape_boost_exponent", [("if (pr.p1 < 1.0) g *= pow(u01(w[3]), 1.0 / pr.p1);",
                                           "if (pr.p1 < 1.0) g *= pow(u01(w[3]), pr.p1);")],
     [P.test_prior_draw_distributions]),
    ("log_uniform_drawn_uniform", [("return log(pr.p1) + (log(pr.p2) - log(pr.p1)) * u01(w[0]);",
                                    "return log(pr.p1 + (pr.p2 - pr.p1) * u01(w[0]));")],
     [P.test_prior_draw_distributions]),
    ("gamma_log_prior_rate_sign", [("case PR_GAMMA: return (pr.p1 - 1.0) * log(u) - pr.p2 * u;",
                                    "case PR_GAMMA: return (pr.p1 - 1.0) * log(u) + pr.p2 * u;")],
     [P.test_mh_keeps_prior_at_beta_zero, P.test_evidence_k1_quadrature_gamma_amplitude]),
    ("normal_log_prior_dropped", [("return -0.5 * z * z;", "return 0.0;")],
     [P.test_mh_keeps_gaussian_posterior_invariant, P.test_evidence_linear_gaussian_closed_form]),
    # tempering (Eq. (10)) and the evidence (Eq. (11))
    ("ess_not_a_fraction", [("return s1 * s1 / ((double)T * s2);", "return s1 * s1 / s2;")],
     [P.test_ess_limits_and_monotonicity]),
    ("bisection_returns_upper_end", [("return lo > 0.0 ? lo : hi;", "return hi;")],
     [P.test_bisection_bracket_property]),
    ("bisection_branches_swapped", [("            lo = mid;\n        else\n            hi = mid;",
                                     "            hi = mid;\n        else\n            lo = mid;")],
     [P.test_bisection_bracket_property, P.test_bisection_exponential_closed_form]),
    ("final_step_never_taken", [("if (orc_ess_frac(e, T, room) >= rho) {", "if (0) {")],
     [P.test_bisection_final_step_when_flat, P.test_flat_likelihood_single_stage]),
    ("bisection_stop_absolute", [("hi - lo > 1e-7 * hi", "hi - lo > 1e-7")],
     [P.test_bisection_bracket_property, P.test_bisection_exponential_closed_form]),
    ("evidence_mean_not_taken", [("logz += -delta * emin + log(sw / (double)Tc);",
                                  "logz += -delta * emin + log(sw);")],
     [P.test_evidence_linear_gaussian_closed_form]),
    ("evidence_shift_dropped", [("logz += -delta * emin + log(sw / (double)Tc);",
                                 "logz += log(sw / (double)Tc);")],
     [P.test_evidence_linear_gaussian_closed_form]),
    ("beta_not_accumulated", [("beta = final_step ? 1.0 : beta + delta;", "beta = final_step ? 1.0 : delta;")],
     [P.test_evidence_linear_gaussian_closed_form]),
    # systematic resampling on integer weights
    ("quantise_scale", [("q[i] = (uint64_t)floor(ldexp(w[i], 40));", "q[i] = (uint64_t)floor(ldexp(w[i], 32));")],
     [P.test_quantise_is_exact]),
    ("resample_offset_dropped", [
        ("unsigned __int128 t = ((unsigned __int128)m * Q + r) / (unsigned __int128)M;",
         "unsigned __int128 t = ((unsigned __int128)m * Q) / (unsigned __int128)M;")],
     [P.test_resample_matches_textbook_float_version]),
    ("resample_exclusive_prefix", [("while (C <= t) {", "while (C < t) {")],
     [P.test_resample_equal_and_zero_weights_are_exact, P.test_resample_matches_textbook_float_version,
      P.test_resample_offspring_bounds]),
    # Metropolis (Sec. II B 4)
    ("log_uniform_support_in_natural_units", [("case PR_LOG_UNIFORM: return u >= log(pr.p1) && u <= log(pr.p2);",
                                               "case PR_LOG_UNIFORM: return u >= pr.p1 && u <= pr.p2;")],
     [P.test_mh_keeps_prior_at_beta_zero]),
    ("log_uniform_value_not_exponentiated", [("return pr.kind == PR_LOG_UNIFORM ? exp(u) : u; }", "return u; }")],
     [P.test_evidence_k1_tensor_quadrature_all_three_free, P.test_evidence_linear_gaussian_closed_form]),
    ("normal_log_prior_sd_dropped", [("double z = (u - pr.p1) / pr.p2;", "double z = (u - pr.p1);")],
     [P.test_mh_keeps_gaussian_posterior_invariant, P.test_evidence_linear_gaussian_closed_form]),
    ("standard_mode_energy_not_updated", [("            memcpy(u_out + (size_t)m * d, cur, sizeof(double) * d);\n            E_out[m] = Ec;",
                                           "            memcpy(u_out + (size_t)m * d, cur, sizeof(double) * d);\n            E_out[m] = E_start[m];")],
     [P.test_evidence_linear_gaussian_closed_form, P.test_evidence_k1_quadrature_free_centre,
      P.test_evidence_k1_tensor_quadrature_all_three_free]),
    ("standard_mode_keeps_start_state", [("            memcpy(u_out + (size_t)m * d, cur, sizeof(double) * d);\n            E_out[m] = Ec;",
                                          "            memcpy(u_out + (size_t)m * d, u_start + (size_t)m * d, sizeof(double) * d);\n            E_out[m] = E_start[m];")],
     [P.test_evidence_linear_gaussian_closed_form, P.test_evidence_k1_quadrature_free_centre,
      P.test_evidence_k1_tensor_quadrature_all_three_free]),
    ("mh_energy_difference_reversed", [("if (log(u01(ww[2])) < -beta * (Ep - Ec) + dlp) {",
                                        "if (log(u01(ww[2])) < -beta * (Ec - Ep) + dlp) {")],
     [P.test_mh_keeps_gaussian_posterior_invariant]),
    ("mh_prior_ratio_dropped", [("< -beta * (Ep - Ec) + dlp) {", "< -beta * (Ep - Ec)) {")],
     [P.test_mh_keeps_prior_at_beta_zero, P.test_mh_keeps_gaussian_posterior_invariant]),
    ("mh_support_check_dropped", [("if (!in_support(c->pri[j], up)) continue;", ";")],
     [P.test_mh_keeps_prior_at_beta_zero]),
    ("mh_rejection_keeps_proposal", [("cur[j] = old;", "(void)old;")],
     [P.test_mh_keeps_prior_at_beta_zero, P.test_mh_keeps_gaussian_posterior_invariant]),
    # step sizes (Sec. II B 4, the lambda x SD rule)
    ("step_sd_unweighted", [
        ("for (int64_t i = 0; i < T; ++i) m1 += w[i] * u[i * d + j];\n        m1 /= sw;",
         "for (int64_t i = 0; i < T; ++i) m1 += u[i * d + j];\n        m1 /= (double)T;"),
        ("v += w[i] * t * t;\n        }\n        v /= sw;", "v += t * t;\n        }\n        v /= (double)T;")],
     [A.test_step_sizes_weighted_sd_by_replication, A.test_first_stage_step_uses_pre_resample_weights]),
    ("step_sizes_after_resampling", [
        ("        orc_step_sizes_ex(job, u, w, Tc, stage > 1 ? rate : NULL, lam, step, hist, beta_prev, beta);\n"
         "        if (out->step_trace)\n"
         "            for (int j = 0; j < d; ++j) out->step_trace[(size_t)stage * d + j] = step[j];\n", ""),
        ("        /* -- Metropolis rejuvenation at beta */\n",
         "        for (int64_t m = 0; m < S; ++m) w[m] = 1.0;\n"
         "        orc_step_sizes_ex(job, us, w, S, stage > 1 ? rate : NULL, lam, step, hist, beta_prev, beta);\n"
         "        if (out->step_trace)\n"
         "            for (int j = 0; j < d; ++j) out->step_trace[(size_t)stage * d + j] = step[j];\n")],
     [A.test_first_stage_step_uses_pre_resample_weights]),
    ("acceptance_update_sign", [("lam[j] *= exp(acc_rate[j] - 0.44);", "lam[j] *= exp(0.44 - acc_rate[j]);")],
     [A.test_step_sizes_lambda_updates_and_clamps, A.test_second_stage_step_follows_acceptance]),
    ("lambda_upper_clamp_dropped", [("if (lam[j] > 10.0) lam[j] = 10.0;", ";")],
     [A.test_step_sizes_lambda_updates_and_clamps]),
    ("step_floor_not_relative", [("double floor_sd = 1e-9 * (1.0 + fabs(m1));", "double floor_sd = 1e-9;")],
     [A.test_step_sizes_floor_for_a_collapsed_component]),
    ("fixed_component_given_a_step", [("            step[j] = 0.0;\n            continue;",
                                       "            step[j] = 1.0;\n            continue;")],
     [A.test_step_sizes_weighted_sd_by_replication]),
    # waste-free SMC (Sec. II B 3)
    ("waste_free_keeps_start_state", [
        ("memcpy(u_out + (size_t)(m * n + t) * d, cur, sizeof(double) * d);\n"
         "                E_out[m * n + t] = Ec;",
         "memcpy(u_out + (size_t)(m * n + t) * d, u_start + (size_t)m * d, sizeof(double) * d);\n"
         "                E_out[m * n + t] = E_start[m];")],
     [A.test_waste_free_keeps_every_post_sweep_state]),
    ("waste_free_keeps_last_sweep_only", [("if (job->waste_free) {\n                memcpy",
                                           "if (job->waste_free && t == n - 1) {\n                memcpy")],
     [A.test_waste_free_keeps_every_post_sweep_state]),
    ("waste_free_reweights_chains_only", [
        ("for (int64_t i = 0; i < Tc; ++i)\n            if (isfinite(E[i]) && E[i] < emin)",
         "for (int64_t i = 0; i < S; ++i)\n            if (isfinite(E[i]) && E[i] < emin)"),
        ("for (int64_t i = 0; i < Tc; ++i) e[i] = isfinite(E[i])", "for (int64_t i = 0; i < S; ++i) e[i] = isfinite(E[i])"),
        ("orc_choose_delta(e, Tc, beta,", "orc_choose_delta(e, S, beta,"),
        ("for (int64_t i = 0; i < Tc; ++i) {\n            w[i] = isfinite(e[i])",
         "for (int64_t i = 0; i < S; ++i) {\n            w[i] = isfinite(e[i])"),
        ("log(sw / (double)Tc);", "log(sw / (double)S);"),
        ("orc_step_sizes_ex(job, u, w, Tc,", "orc_step_sizes_ex(job, u, w, S,"),
        ("orc_quantise(w, Tc, q);", "orc_quantise(w, S, q);"),
        ("orc_resample(q, Tc, S,", "orc_resample(q, S, S,")],
     [A.test_waste_free_second_stage_runs_over_all_states]),
    ("lambda_initial_value", [("for (int j = 0; j < d; ++j) lam[j] = 2.38;", "for (int j = 0; j < d; ++j) lam[j] = 1.0;")],
     [A.test_first_stage_step_uses_pre_resample_weights]),
    ("waste_free_chain_count_floored", [("(T + n - 1) / n : T; /* chains per stage */", "T / n : T; /* chains per stage */")],
     [P.test_waste_free_particle_count]),
    ("run_energy_model_variance_ignored", [("if (job->bg_kind == BG_SHIRLEY || job->noise == NOISE_MODEL)",
                                            "if (job->bg_kind == BG_SHIRLEY)")],
     [P.test_constant_model_variance_reduces_to_known_sigma]),
    ("run_energy_shirley_ignored", [("if (job->bg_kind == BG_SHIRLEY || job->noise == NOISE_MODEL)",
                                     "if (job->noise == NOISE_MODEL)")],
     [P.test_shirley_known_sigma_run_is_exact_at_fixed_parameters]),
    ("run_energy_poisson_ignored", [("if (job->family == FAM_XRD_PHASE || job->noise == NOISE_POISSON)",
                                     "if (job->family == FAM_XRD_PHASE)")],
     [P.test_poisson_counts_with_a_peak_family_fixed_parameters_exact]),
    ("poisson_normaliser_y_sign", [("lognorm += (y > 0.0 ? y * log(y) : 0.0) - y - lgamma(y + 1.0);",
                                    "lognorm += (y > 0.0 ? y * log(y) : 0.0) + y - lgamma(y + 1.0);")],
     [P.test_xrd_poisson_log_z_of_fixed_background_is_exact]),
    ("xrd_background_lorentz_width_doubled", [("xrd_pv(x, bg[1], bg[1], bg[2])", "xrd_pv(x, bg[1], 2.0 * bg[1], bg[2])")],
     [P.test_xrd_background_closed_form]),
    # the history step-size predictor (step_rule 1)
    ("predictor_history_at_next_beta", [("double x = log(beta_prev), y = log(sig);",
                                         "double x = log(beta_next), y = log(sig);")],
     [A.test_predictor_hits_target_rate_on_a_power_law, A.test_predictor_history_weights_and_bounds]),
    ("predictor_target_rate", [("/ tan(M_PI * 0.44 / 2.0);", "/ tan(M_PI * 0.234 / 2.0);")],
     [A.test_predictor_hits_target_rate_on_a_power_law]),
    ("predictor_inversion_factor", [("double sig = s_prev * tan(M_PI * a / 2.0) / 2.0;",
                                     "double sig = s_prev * tan(M_PI * a / 2.0);")],
     [A.test_predictor_hits_target_rate_on_a_power_law]),
    ("predictor_extrapolates_to_previous_beta", [("b * (log(beta_next) - xm)", "b * (log(beta_prev) - xm)")],
     [A.test_predictor_hits_target_rate_on_a_power_law]),
    ("predictor_history_not_halved", [("for (int k = 0; k < 5; ++k) h[k] *= 0.5;", ";")],
     [A.test_predictor_history_weights_and_bounds]),
    ("predictor_slope_not_clamped", [("if (b > 0.0) b = 0.0;", ";")],
     [A.test_predictor_history_weights_and_bounds]),
    ("predictor_upper_bound_dropped", [("if (st > 10.0 * sd_pop) st = 10.0 * sd_pop;", ";")],
     [A.test_predictor_history_weights_and_bounds]),
]


# Mistakes in the Python half of the oracle (the cross-K post-processing):
# (name, function, edits, pins).
PY_MUTANTS = [
    ("posterior_not_normalised", "posterior_over_k", [("return p / p.sum()", "return p")],
     [P.test_posterior_over_k_is_softmax_of_evidence]),
    ("posterior_without_max_shift", "posterior_over_k", [("p = np.exp(lz - m)", "p = np.exp(lz)")],
     [P.test_posterior_over_k_survives_large_evidences]),
    ("summary_sorted_by_amplitude", "sorted_summary", [("peaks[:, :, 1]", "peaks[:, :, 0]")],
     [P.test_sorted_summary_orders_peaks_by_centre]),
    ("summary_pv_read_as_three_components", "sorted_summary",
     [("p = 4 if family == 2 else 3", "p = 3")], [P.test_sorted_summary_orders_peaks_by_centre]),
    ("summary_sorts_phases", "sorted_summary", [("if family == 4:", "if family == -1:")],
     [P.test_sorted_summary_orders_peaks_by_centre]),
]


def _mutated_source(src: str, edits) -> str:
    for e in edits:
        old, new = e[0], e[1]
        count = e[2] if len(e) > 2 else 1
        found = src.count(old)
        assert found == count, f"planted edit expects {count} occurrence(s), found {found}: {old!r}"
        src = src.replace(old, new)
    return src


@pytest.fixture(scope="module")
def mutant_libs():
    """Every mutant built once (gcc in parallel), by name."""
    with open(oracle.source()) as fh:
        base = fh.read()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")

    def build(m):
        name, edits, _ = m
        src = os.path.join(tmp, f"{name}.c")
        with open(src, "w") as fh:
            fh.write(_mutated_source(base, edits))
        return name, oracle.compile_library(src, os.path.join(tmp, f"lib{name}.so"))

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        paths = dict(ex.map(build, MUTANTS))
    yield paths
    for name, path in paths.items():
        for f in (path, os.path.join(tmp, f"{name}.c")):
            if os.path.exists(f):
                os.remove(f)
    os.rmdir(tmp)


def _calls(fn):
    """The argument tuples a test function is collected with (one
    parametrize mark at most)."""
    marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
    if not marks:
        return [()]
    assert len(marks) == 1
    names, values = marks[0].args[0], marks[0].args[1]
    n = len(names.split(",")) if isinstance(names, str) else len(names)
    return [tuple(v) if n > 1 else (v,) for v in values]


def _detects(fn) -> bool:
    assert not [p for p in inspect.signature(fn).parameters
                if p not in set(itertools.chain.from_iterable(
                    m.args[0].split(",") if isinstance(m.args[0], str) else m.args[0]
                    for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"))]
    for args in _calls(fn):
        try:
            fn(*args)
        except AssertionError:
            return True
    return False


def test_pins_pass_on_the_oracle_itself():
    """The harness calls the pins the way pytest does: on the unmutated
    oracle none of them fails."""
    pins = [f for m in MUTANTS + PY_MUTANTS for f in m[-1]]
    for fn in {id(f): f for f in pins}.values():
        assert not _detects(fn), fn.__name__


@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(mutant, mutant_libs):
    name, _, pins = mutant
    oracle.use_library(oracle.bind(C.CDLL(mutant_libs[name])))
    try:
        caught = next((fn.__name__ for fn in pins if _detects(fn)), None)
    finally:
        oracle.use_library(None)
    assert caught, f"mistake '{name}' passed {[f.__name__ for f in pins]}"


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a mutant's overflow / 0/0 is its failure
@pytest.mark.parametrize("mutant", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_python_mistake_fails_a_pin(mutant):
    name, func, edits, pins = mutant
    original = getattr(oracle, func)
    src = _mutated_source(textwrap.dedent(inspect.getsource(original)), edits)
    ns = dict(vars(oracle))
    exec(compile(src, f"<oracle mutant {name}>", "exec"), ns)
    setattr(oracle, func, ns[func])
    try:
        caught = next((fn.__name__ for fn in pins if _detects(fn)), None)
    finally:
        setattr(oracle, func, original)
    assert caught, f"mistake '{name}' passed {[f.__name__ for f in pins]}"
