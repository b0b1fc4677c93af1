"""The oracle's pins catch plausible mistakes: each case plants one mistake
in a copy of oracle/orc.cpp (a sign, a coefficient, a transposed index, a
dropped condition), builds it into a separate library and runs the pin that
should fail against it (in a subprocess, through ORC_LIB).  The unmodified
oracle passes the same pins in test_oracle_pins.py.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "orc.cpp")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# id: (text in orc.cpp, its mistaken replacement, the pin that must fail)
MUTATIONS = {
    "roe_left_eigenvector_sign": ("0.5 * (b2 + un * ic), 0.5 * (-b1 * un - ic)",
                                  "0.5 * (b2 - un * ic), 0.5 * (-b1 * un - ic)",
                                  "test_eigensystem_inverse_and_roe_property"),
    "hllc_star_energy_sign": ("(Ss - q.vel[0]) * (Ss + q.p / mK)", "(Ss - q.vel[0]) * (Ss - q.p / mK)",
                              "test_hllc_exact_on_isolated_shocks"),
    "hllc_contact_speed": ("(((b.p - a.p) + uL * mL) - uR * mR)", "(((b.p - a.p) + uL * mL) + uR * mR)",
                           "test_hllc_exact_on_isolated_shocks"),
    "llf_not_everywhere": ("if (flux == FLUX_ROE && lL > 0.0 && lR > 0.0 && lt > 0.0) {",
                           "if (lL > 0.0 && lR > 0.0 && lt > 0.0) {",
                           "test_llf_face_flux_on_a_step_closed_form"),
    "llf_speed_from_roe_average": ("      T alpha = omax(oabs(lL), oabs(lR));\n      T fp[6], fm[6];",
                                   "      T alpha = oabs(lt);\n      T fp[6], fm[6];",
                                   "test_roe_llf_switch_on_a_transonic_step_closed_form"),
    "coarsen_ignores_parent_detail": ("          if (dpar[pk | (inst << 56)] > ep) all = false;",
                                      "          if (dpar[pk | (inst << 56)] > 1e300 * ep) all = false;",
                                      "test_refined_groups_are_not_coarsened_right_away"),
    "weno5_linear_weights": ("  T a1 = 0.6 / ((eps + beta1) * (eps + beta1));\n  T a2 = 0.3 / ((eps + beta2) * (eps + beta2));\n  T sum = (a0 + a1) + a2;\n  T q0",
                             "  T a1 = 0.5 / ((eps + beta1) * (eps + beta1));\n  T a2 = 0.4 / ((eps + beta2) * (eps + beta2));\n  T sum = (a0 + a1) + a2;\n  T q0",
                             "test_fifth_order_convergence_density_wave[0-0]"),
    "teno5_cutoff": ("const double eps = 1e-40, CT = 1e-5;", "const double eps = 1e-40, CT = 1e-1;",
                     "test_teno5_matches_its_definition"),
    "morton_negative_carry": ("f = (sign > 0) ? (nbit | f) : ((!nbit) | f);", "f = (sign > 0) ? (nbit | f) : (nbit | f);",
                              "test_morton_neighbours_brute_force"),
    "jump_face_mean": ("double val = 0.25 * ((f(0, 0) + f(1, 0)) + (f(0, 1) + f(1, 1)));",
                       "double val = 0.25 * ((f(0, 0) + f(1, 0)) + (f(0, 1) + f(0, 1)));",
                       "test_conservation_periodic_with_jumps"),
    "hllc_no_fallback": ("    if (!admissible(UL, g, B) || !admissible(UR, g, B)) {\n      for (int j = 0; j < 5; ++j) {\n        UL[j] = Ur[2][j];",
                         "    if (false) {\n      for (int j = 0; j < 5; ++j) {\n        UL[j] = Ur[2][j];",
                         "test_hllc_inadmissible_face_state_falls_back_to_the_cells"),
    "detail_relative_to_prediction": ("double r = std::fabs(uf - pr) / std::fabs(uf);",
                                      "double r = std::fabs(uf - pr) / std::fabs(pr);",
                                      "test_detail_norm_of_a_single_perturbed_cell"),
    "detail_without_halo": ("        if (ghost) continue;\n        for (int vi = 0; vi < 2; ++vi) {",
                            "        if (ghost || sx || sy || sz) continue;\n        for (int vi = 0; vi < 2; ++vi) {",
                            "test_detail_norm_of_a_single_perturbed_cell"),
    "rk3_weights": ("const double RK_B3[3] = {1.0, 0.25, 2.0 / 3.0};", "const double RK_B3[3] = {1.0, 0.3, 2.0 / 3.0};",
                    "test_fifth_order_convergence_density_wave[0-0]"),
    "projection_weight": ("P.u[(size_t)v2 * NCELL + sidx(I, J, K)] = 0.125 * (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c7)));",
                          "P.u[(size_t)v2 * NCELL + sidx(I, J, K)] = 0.125 * (((c0 + c1) + (c2 + c3)) + ((c4 + c5) + (c6 + c6)));",
                          "test_projection_is_the_mean_of_the_children"),
    "gravity_work_sign": ("n.L[(size_t)4 * NINT + t] = n.L[(size_t)4 * NINT + t] + ((mx * gx + my * gy) + mz * gz);",
                          "n.L[(size_t)4 * NINT + t] = n.L[(size_t)4 * NINT + t] - ((mx * gx + my * gy) + mz * gz);",
                          "test_gravity_source_term"),
    "wenoao_quartic_smoothness": ("(781.0 / 20.0) * (u3 * u3)", "(781.0 / 30.0) * (u3 * u3)",
                                  "test_wenoao_matches_its_definition"),
    "wenoao_weight_exponent": ("T w5 = g5 * (1.0 + r5 * r5)", "T w5 = g5 * (1.0 + r5)",
                               "test_wenoao_matches_its_definition"),
    "viscous_stress_not_symmetrised": ("tau[i] = mu * (G[i][d] + G[d][i]);", "tau[i] = mu * (G[i][d] + G[i][d]);",
                                       "test_viscous_terms_on_a_linear_velocity_field"),
    "viscous_bulk_term_sign": ("tau[d] = tau[d] - ((2.0 / 3.0) * mu) * div;",
                               "tau[d] = tau[d] + ((2.0 / 3.0) * mu) * div;",
                               "test_viscous_terms_on_a_linear_velocity_field"),
    "prediction_coefficient": ("const double C0 = -22.0 / 128.0, C1 = 3.0 / 128.0;",
                               "const double C0 = -22.0 / 128.0, C1 = -3.0 / 128.0;",
                               "test_prediction_reproduces_quartics"),
    "cfl_abs_of_sum": ("std::fabs(q.vel[d]) + q.c);", "std::fabs(q.vel[d] + q.c));",
                       "test_cfl_time_step_closed_form[0.0]"),
    "cfl_viscous_factor": ("((6.0 * C.c.mu) * ir[i])", "((2.0 * C.c.mu) * ir[i])",
                           "test_cfl_time_step_closed_form[0.05]"),
    "symmetry_mirror_index": ("else src[d] = (side == 0) ? (-1 - a) : (2 * NB - 1 - a);",
                              "else src[d] = (side == 0) ? (-a) : (2 * NB - 1 - a);",
                              "test_symmetry_walls_are_the_mirror_image[0-0]"),
    "symmetry_flips_x_momentum": ("if (bc == BC_SYMMETRY && v == 1 + d) val = -val;",
                                  "if (bc == BC_SYMMETRY && v == 1) val = -val;",
                                  "test_symmetry_walls_are_the_mirror_image[1-2]"),
    "face_average_top_down": ("void average_faces(Ctx& C) {\n  int lm = max_level(C);\n  for (int l = lm - 1; l >= 0; --l) {",
                              "void average_faces(Ctx& C) {\n  int lm = max_level(C);\n  for (int l = 0; l < lm; ++l) {",
                              "test_conservation_across_two_level_jumps"),
    "level_threshold_dimension": ("double el = std::ldexp(C.c.eps, -3 * (lmx - n.level));",
                                  "double el = std::ldexp(C.c.eps, -2 * (lmx - n.level));",
                                  "test_level_thresholds_decide_the_tags"),
    "level_threshold_of_parent": ("double el = std::ldexp(C.c.eps, -3 * (lmx - n.level));",
                                  "double el = std::ldexp(C.c.eps, -3 * (lmx - (n.level - 1)));",
                                  "test_level_thresholds_decide_the_tags"),
    "child_coordinate_bits": ("for (int d = 0; d < 3; ++d) c.X[d] = 2 * P.X[d] + ((ch >> d) & 1);",
                              "for (int d = 0; d < 3; ++d) c.X[d] = 2 * P.X[d] + ((ch >> (2 - d)) & 1);",
                              "test_refinement_puts_each_prediction_in_its_octant"),
    "halo_predicted_from_wrong_octant": ("val = predict_cell(&par->u[(size_t)v * NCELL], ch, i, j, k);",
                                         "val = predict_cell(&par->u[(size_t)v * NCELL], ch ^ 1, i, j, k);",
                                         "test_halo_fill_is_exact_on_a_quartic_with_jumps"),
    "halo_fill_fine_to_coarse": ("  for (int l = 0; l <= lm; ++l) {\n    std::vector<Node*> v = nodes_at(C, l, false);\n#pragma omp parallel for schedule(dynamic)\n    for (long t = 0; t < (long)v.size(); ++t) fill_node(",
                                 "  for (int l = lm; l >= 0; --l) {\n    std::vector<Node*> v = nodes_at(C, l, false);\n#pragma omp parallel for schedule(dynamic)\n    for (long t = 0; t < (long)v.size(); ++t) fill_node(",
                                 "test_halo_fill_is_exact_on_a_quartic_with_jumps"),
    "sibling_lookup_drops_instance": ("uint64_t sk = ((pk << 3) | (uint64_t)c) | (inst << 56);",
                                      "uint64_t sk = ((pk << 3) | (uint64_t)c);",
                                      "test_instances_evolve_independently"),
    "weno5_smoothness_coefficient": ("T weno5(T a, T b, T c, T d, T e) {\n  const double eps = 1e-6;\n  T t1 = (a - 2.0 * b) + c, t2 = (a - 4.0 * b) + 3.0 * c;\n  T beta0 = (13.0 / 12.0) * t1 * t1 + 0.25 * t2 * t2;",
                                     "T weno5(T a, T b, T c, T d, T e) {\n  const double eps = 1e-6;\n  T t1 = (a - 2.0 * b) + c, t2 = (a - 4.0 * b) + 3.0 * c;\n  T beta0 = (13.0 / 12.0) * t1 * t1 + 0.5 * t2 * t2;",
                                     "test_weno5_matches_its_definition"),
    "weno5_eps": ("T weno5(T a, T b, T c, T d, T e) {\n  const double eps = 1e-6;",
                  "T weno5(T a, T b, T c, T d, T e) {\n  const double eps = 1e-40;",
                  "test_weno5_matches_its_definition"),
    "detail_norm_reads_momentum": ("const int vars[2] = {0, 4};", "const int vars[2] = {0, 1};",
                                   "test_detail_norm_of_a_single_perturbed_cell"),
    "viscous_limit_takes_max_rho": ("ir[n.inst] = std::max(ir[n.inst], 1.0 / q.rho);", "ir[n.inst] = std::max(ir[n.inst], q.rho);",
                                    "test_cfl_time_step_closed_form[0.05]"),
    "stiffened_pressure_offset": ("q.p = (g - 1.0) * (U[4] - 0.5 * q.rho * q2) - g * B;",
                                  "q.p = (g - 1.0) * (U[4] - 0.5 * q.rho * q2) - B;",
                                  "test_cfl_time_step_closed_form[0.0]"),
    "hllc_left_speed_without_roe": ("T SL = omin(uL - a.c, e.lam[0]);", "T SL = uL - a.c;",
                                    "test_hllc_exact_on_isolated_shocks[0]"),
    "rhs_y_faces_transposed": ("acc = acc + (F[fidx(1, v, j, i, k)] - F[fidx(1, v, j + 1, i, k)]);",
                               "acc = acc + (F[fidx(1, v, j, k, i)] - F[fidx(1, v, j + 1, k, i)]);",
                               "test_rhs_commutes_with_rotations_and_mirrors[rotate-0-0-0.0]"),
    "tangential_momenta_swapped": ("  U[1 + rot_axis(d, 1)] = R[2];\n  U[1 + rot_axis(d, 2)] = R[3];",
                                   "  U[1 + rot_axis(d, 1)] = R[3];\n  U[1 + rot_axis(d, 2)] = R[2];",
                                   "test_rhs_commutes_with_rotations_and_mirrors[mirror-0-0-0.0]"),
    "level1_groups_coarsened": ("} else if (n.level >= 2) {", "} else if (n.level >= 1) {",
                                "test_tags_uniform_state_collapses_to_level1"),
    "feature_alpha_from_roe_average": ("    double alpha = std::max(std::fabs(lL), std::fabs(lR));\n    for (int m = 0; m < 5; ++m) {",
                                       "    double alpha = std::fabs(e.lam[k]);\n    for (int m = 0; m < 5; ++m) {",
                                       "test_selector_features_with_the_split_active_match_their_definition[0]"),
    "feature_without_alpha_term": ("compress_diff(sgn * (std::fabs(dg) + alpha * std::fabs(dv)));",
                                   "compress_diff(sgn * std::fabs(dg));",
                                   "test_selector_features_with_the_split_active_match_their_definition[1]"),
    "feature_compression_constant": ("double a = std::log10(1.0 + 1e6 * std::fabs(d)) / 8.0;",
                                     "double a = std::log10(1.0 + 1e5 * std::fabs(d)) / 8.0;",
                                     "test_selector_features_with_the_split_active_match_their_definition[2]"),
    "lts_schedule": ("      if (r % (1 << (L - l)) != 0) continue;\n      if (nodes_at(C, l, false).empty()) continue;",
                     "      if (r % (1 << l) != 0) continue;\n      if (nodes_at(C, l, false).empty()) continue;",
                     "test_lts_density_wave_crosses_a_jump"),
    "lts_no_reflux": ("  average_fmac(C);\n  lts_reflux(C);\n  project(C);", "  average_fmac(C);\n  project(C);",
                      "test_lts_conserves_across_jumps[3]"),
    "lts_frozen_coarse_levels": ("            n.u[si] = (1.0 - th) * n.un[ii] + th * n.u[si];",
                                 "            n.u[si] = n.un[ii];",
                                 "test_lts_density_wave_crosses_a_jump"),
    "lts_stage_flux_weights": ("const double RK_W3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};",
                               "const double RK_W3[3] = {1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0};",
                               "test_lts_conserves_across_jumps[2]"),
    "rk2_weights": ("const double RK_B2[2] = {1.0, 0.5};", "const double RK_B2[2] = {1.0, 0.6};",
                    "test_rk2_is_second_order_in_time"),
}


def _run_pin(so, pin, threads):
    env = dict(os.environ, ORC_LIB=so, OMP_NUM_THREADS=str(threads))
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", f"{PINS}::{pin}"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Build every mutant, then run each one's pin, all concurrently."""
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {}
    for mid, (old, new, _) in MUTATIONS.items():
        assert src.count(old) == 1, mid
        p = os.path.join(d, mid + ".cpp")
        open(p, "w").write(src.replace(old, new))
        jobs[mid] = (p, os.path.join(d, mid + ".so"))
    ncpu = os.cpu_count() or 1
    with cf.ThreadPoolExecutor(max_workers=min(8, ncpu)) as ex:
        list(ex.map(lambda j: oracle.compile_to(*j), jobs.values()))
    workers = min(len(MUTATIONS), max(1, ncpu // 2))
    threads = max(1, ncpu // workers)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {mid: ex.submit(_run_pin, jobs[mid][1], MUTATIONS[mid][2], threads) for mid in MUTATIONS}
        return {mid: f.result() for mid, f in futs.items()}


@pytest.mark.parametrize("mid", sorted(MUTATIONS))
def test_pin_catches_planted_mistake(outcomes, mid):
    r = outcomes[mid]
    assert r.returncode == 1, (mid, MUTATIONS[mid][2], r.stdout[-2000:])
    assert "failed" in r.stdout, (mid, r.stdout[-2000:])
