"""The pins are not vacuous: plant a mistake in a copy of the oracle (on the
CPU) and check that the pin aimed at it fails.

Each entry replaces one line of the oracle's C source by a plausible slip
(a flipped sign, a dropped term, a transposed index, a wrong constant) and
names the pin tests that must catch it.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
T = "tests/test_oracle_pins.py::"

MUTATIONS = {
    "dissipation_sign": ("double dq = lam * (eps2 * D1 - eps4 * D3);",
                         "double dq = lam * (eps2 * D1 + eps4 * D3);",
                         ["test_fourth_difference_mode_decays"]),
    "heat_flux_sign": ("double qx = -kap * gr[3][0]", "double qx = kap * gr[3][0]",
                       ["test_heat_conduction_sign_and_rate"]),
    "eta_metric_row": ("M[3 * N + nn] = J * (y_zeta * z_xi - y_xi * z_zeta);",
                       "M[3 * N + nn] = J * (y_eta * z_xi - y_xi * z_eta);",
                       ["test_metric_identity"]),
    "stokes_two_thirds": ("double txx = mu * (2.0 * gr[0][0] - (2.0 / 3.0) * div);",
                          "double txx = mu * (2.0 * gr[0][0] - (1.0 / 3.0) * div);",
                          ["test_manufactured_solution_second_order"]),
    "beta_transposed": ("double bx = txx * uf + txy * vf + txz * wf - qx;",
                        "double bx = txx * uf + txy * wf + txz * vf - qx;",
                        ["test_manufactured_solution_second_order"]),
    "rk_alpha3": ("3.0 / 8.0, 1.0 / 2.0", "3.0 / 7.0, 1.0 / 2.0",
                  ["test_rk5_amplification_polynomial",
                   "test_runge_kutta_coefficients_and_stability_statement"]),
    "closure_sign": ("double Dm = (am >= 0) ? W_of(S, a, q) - W_of(S, am, q) : -D1;",
                     "double Dm = (am >= 0) ? W_of(S, a, q) - W_of(S, am, q) : D1;",
                     ["test_fourth_difference_boundary_closure"]),
    "lbar_ratio": ("S->lbar[1][n] = l[1] * (1.0 + sqrt(l[0] / l[1]) + sqrt(l[2] / l[1]));",
                   "S->lbar[1][n] = l[1] * (1.0 + sqrt(l[0] / l[1]) + sqrt(l[1] / l[2]));",
                   ["test_fourth_difference_mode_decays"]),
    "tangential_sum": ("dphi[q][t] = 0.25 * ((phi[q][ap] - phi[q][amt]) +",
                       "dphi[q][t] = 0.25 * ((phi[q][ap] - phi[q][amt]) -",
                       ["test_manufactured_solution_second_order"]),
    "riemann_plus": ("double Rp = qne + 2.0 * a_e / gm1;", "double Rp = qne - 2.0 * a_e / gm1;",
                     ["test_far_field_keeps_free_stream"]),
    "far_field_exit_source_node": (
        "if (riemann_far_field(gam, rho, u, v, w, p, ex * inv, ey * inv, ez * inv, q))\n"
        "        for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + ne];",
        "if (riemann_far_field(gam, rho, u, v, w, p, ex * inv, ey * inv, ez * inv, q))\n"
        "        for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + nf];",
        ["test_far_field_supersonic_branches"]),
    "far_field_inflow_pressure": ("cons_from(gam, rho_inf, 0.0, 0.0, 0.0, p_inf, q);",
                                  "cons_from(gam, rho_inf, 0.0, 0.0, 0.0, 1.0, q);",
                                  ["test_far_field_supersonic_branches",
                                   "test_characteristic_entrance_supersonic_branches"]),
    "far_field_sonic_exit_edge": ("if (Mn >= 1.0) {", "if (Mn > 1.0) {",
                                  ["test_characteristic_entrance_supersonic_branches"]),
    "entrance_exit_source_node": ("                              -ez * inv, q))\n"
                                  "          for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + ne];",
                                  "                              -ez * inv, q))\n"
                                  "          for (int c = 0; c < 5; ++c) q[c] = Qs[c * N + n];",
                                  ["test_characteristic_entrance_supersonic_branches"]),
    "energy_flux_p": ("F[4] = Jinv * ((S->Q[4 * N + n] + p) * Th);",
                      "F[4] = Jinv * ((S->Q[4 * N + n]) * Th);",
                      ["test_one_dimensional_jst_reduction"]),
    "face_sensor": ("return fabs(pp - 2.0 * p0 + pm) / (pp + 2.0 * p0 + pm);\n  }",
                    "return fabs(pp - 2.0 * p0 + pm) / (pp + p0 + pm);\n  }",
                    ["test_one_dimensional_jst_reduction"]),
    "conservative_outer_swap": ("double cof = product_deriv(&g, xyz, shift, c, t, p, s, q) -",
                                "double cof = product_deriv(&g, xyz, shift, c, s, p, s, q) -",
                                ["test_conservative_metrics_exact_on_affine_grid"]),
    "conservative_period_shift": ("if (w[d] >= g->n[d]) { w[d] -= g->n[d]; v += shift[3 * d + comp]; }",
                                  "if (w[d] >= g->n[d]) { w[d] -= g->n[d]; }",
                                  ["test_conservative_metrics_converge_on_the_periodic_box"]),
    "conservative_face_formula": ("return 0.5 * (-3.0 * metric_product(g, xyz, shift, a, p, s, q) +",
                                  "return 0.5 * (-2.0 * metric_product(g, xyz, shift, a, p, s, q) +",
                                  ["test_conservative_metrics_exact_on_affine_grid"]),
    "local_step_index": ("double h = dtn ? dtn[n] : dt;", "double h = dtn ? dtn[0] : dt;",
                         ["test_rk5_local_steps_per_node"]),
    "local_step_radii": ("dtn[n] = P->cfl / (S.lam[0][n] + S.lam[1][n] + S.lam[2][n]);",
                         "dtn[n] = P->cfl / (S.lam[0][n] + S.lam[1][n] + S.lam[1][n]);",
                         ["test_local_time_steps_closed_form"]),
    "entrance_normal_sign": ("if (riemann_far_field(gam, rho, ue, ve, we, p, -ex * inv, -ey * inv,",
                             "if (riemann_far_field(gam, rho, ue, ve, we, p, ex * inv, -ey * inv,",
                             ["test_characteristic_entrance_above_the_jet"]),
    "subsonic_jet_total_T": ("double Tt = 1.0 + 0.5 * gm1 * P->Mj * P->Mj;",
                             "double Tt = 1.0 + 0.5 * gm1 * P->Mj;",
                             ["test_subsonic_jet_characteristic_entrance"]),
    "dynamic_trace_term": ("double numC = LS - Lkk * trS / 3.0;", "double numC = LS;",
                           ["test_dynamic_procedure_pure_shear_and_dilatation"]),
    "dynamic_test_width": ("Dh2 = 4.0 * D2;", "Dh2 = 2.0 * D2;",
                           ["test_dynamic_procedure_linear_fields_closed_form"]),
    "leonard_favre": ("L[i][j] = L[j][i] = fh[(5 + k) * N + n] - mh[i] * mh[j] / rh;",
                      "L[i][j] = L[j][i] = fh[(5 + k) * N + n] - mh[i] * mh[j];",
                      ["test_dynamic_procedure_linear_fields_closed_form"]),
    "yoshizawa_sign": ("    txx -= iso;", "    txx += iso;",
                       ["test_yoshizawa_isotropic_stress_in_the_residual"]),
    "filter_faces": ("return off == 0 ? 1.0 : 0.0;", "return off == 0 ? 0.5 : 0.25;",
                     ["test_test_filter_transfer_function_and_faces"]),
    "functional_face_row": ("double ex = M[3 * N + n], ey = M[4 * N + n], ez = M[5 * N + n];",
                            "double ex = M[0 * N + n], ey = M[1 * N + n], ez = M[2 * N + n];",
                            ["test_surface_functional_ring_area_closed_form"]),
    "functional_reference_p": ("double dp = p - 1.0 / gam;", "double dp = p - 1.0;",
                               ["test_surface_functional_ring_area_closed_form"]),
    "sutherland_constant": ("double S = 110.4 / P->T_ref;", "double S = 110.0 / P->T_ref;",
                            ["test_paper_constants_are_the_defaults"]),
    "axis_unscaled_storage": ("double J = (Jinv == 0.0) ? 1.0 : 1.0 / Jinv;",
                              "double J = 1.0 / Jinv;",
                              ["test_axis_grid_metrics"]),
    "axis_radii_copy": ("    if (S->M[9 * N + n] != 0.0) continue;\n    int c[3];\n    unlin(&S->g, (size_t)n, c);\n    int c1[3] = {c[0], 1, c[2]};",
                        "    continue;\n    int c[3];\n    unlin(&S->g, (size_t)n, c);\n    int c1[3] = {c[0], 1, c[2]};",
                        ["test_axis_free_stream_preservation"]),
    "axis_plain_mean": ("if (!P->axis && Ja != 0.0 && Jb != 0.0) {", "if (Ja != 0.0 && Jb != 0.0) {",
                        ["test_axis_residual_converges"]),
    "axis_sgs_own": ("double mu_s = sm / (double)nk_;", "double mu_s = mus[n];",
                     ["test_axis_viscosity_is_the_ring_mean"]),
    "axis_exit_normal": ("size_t nm = (M[9 * N + nx_] == 0.0) ? ID(ni - 1, 1, k) : nx_;",
                         "size_t nm = nx_;",
                         ["test_axis_supersonic_exit"]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new, targets = MUTATIONS[name]
    src = open(os.path.join(ROOT, "oracle", "les_oracle.c")).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} vanished"
    for d in ("oracle", "tests", "paper_2301_00817_gb300"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "__pycache__", "csrc"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), tmp_path / "pytest.ini")
    (tmp_path / "oracle" / "les_oracle.c").write_text(src.replace(old, new, 1))
    ids = [T + t for t in targets]
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *ids],
                       cwd=tmp_path, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, r.stdout[-2000:]
