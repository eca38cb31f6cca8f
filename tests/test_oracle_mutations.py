"""The pins bite: plant a plausible mistake in a copy of the oracle source,
build it, and check that at least one pin fails on it (CPU only).

Each entry replaces one line of ls_oracle.c (a dropped term, a wrong sign, a
wrong index, a transposed operand, a wrong rounding) and names the pin
expected to catch it.
"""
import os

import pytest

import oracle as oracle_pkg
import test_oracle_bicgstab as tbs
import test_oracle_block_cg as tbc
import test_oracle_block_cg_deflated as tbd
import test_oracle_block_gmres as tbg
import test_oracle_cg as tcg
import test_oracle_cholesky as tch
import test_oracle_ge_quant as tgq
import test_oracle_gauss_seidel as tgs
import test_oracle_gemv as tgv
import test_oracle_gmres as tgm
import test_oracle_golden as tgo
import test_oracle_jacobi as tja
import test_oracle_mixed as tmx

MUTATIONS = {
    "cg_beta_sign": ("p[i] = r[i] + beta * p[i];", "p[i] = r[i] - beta * p[i];",
                     lambda o: tcg.test_cg_krylov_optimality(o)),
    "cg_alpha": ("double alpha = rho / pq;", "double alpha = rho / (pq * 1.0000001);",
                 lambda o: tcg.test_cg_krylov_optimality(o)),
    "gemv_transposed": ("for (int j = 0; j < ncols; j++) s += a[j] * x[j];",
                        "for (int j = 0; j < ncols; j++) s += A[(long)j * lda + i] * x[j];",
                        lambda o: tgm.test_gmres_matches_lapack(o, 64)),
    "gemv_right_to_left": ("for (int j = 0; j < ncols; j++) s += a[j] * x[j];",
                           "for (int j = ncols - 1; j >= 0; j--) s += a[j] * x[j];",
                           lambda o: tgv.test_rows_summed_left_to_right(o)),
    "residual_sign": ("for (int i = 0; i < n; i++) r[i] = b[i] - r[i];",
                      "for (int i = 0; i < n; i++) r[i] = r[i] - b[i];",
                      lambda o: tgv.test_residual_exact_on_integers(o)),
    "givens_g_sign": ("g[k + 1] = -sn[k] * g[k];", "g[k + 1] = sn[k] * g[k];",
                      lambda o: tgm.test_gmres_minimal_residual(o)),
    "givens_rot_sign": ("HR(j + 1, k) = -sn[j] * a + cs[j] * c;",
                        "HR(j + 1, k) = sn[j] * a + cs[j] * c;",
                        lambda o: tgm.test_gmres_minimal_residual(o)),
    "mgs_drops_last": ("for (int j = 0; j <= k; j++) {                  /* MGS */",
                       "for (int j = 0; j < k; j++) {                  /* MGS */",
                       lambda o: tgm.test_arnoldi_relation_and_orthonormality(o, 12)),
    "backsolve_index": ("for (int j = i + 1; j < k; j++) s -= HR(i, j) * y[j];",
                        "for (int j = i + 1; j < k; j++) s -= HR(j, i) * y[j];",
                        lambda o: tgm.test_gmres_minimal_residual(o)),
    "ge_no_pivoting": ("if (a > best) { best = a; v = i; }", "if (0) { best = a; v = i; }",
                       lambda o: tgq.test_ge_pivoting_and_singular(o)),
    "round_truncates": ("static double round_to_quantum(double d, double q) { return rint(d / q) * q; }",
                        "static double round_to_quantum(double d, double q) { return trunc(d / q) * q; }",
                        lambda o: tgq.test_bf16_nearest_and_ties_to_even(o)),
    "e4m3_bias": ("return s | (uint8_t)((ex + 7) << 3) | (uint8_t)mant;",
                  "return s | (uint8_t)((ex + 6) << 3) | (uint8_t)mant;",
                  lambda o: tgq.test_fp8_quant_row_scales(o)),
    "fcg_no_orthogonalisation": ("double c = dot(n, z, W + (long)j * n) / pw[j];",
                                 "double c = 0.0 * dot(n, z, W + (long)j * n) / pw[j];",
                                 lambda o: tmx.test_fcg_ill_conditioned_bf16(o)),
    "inner_beta_inverted": ("float beta = rho_new / rho;", "float beta = rho / rho_new;",
                            lambda o: tmx.test_inner_cg_f32_solves_stored_matrix(o)),
    "bicgstab_omega_sign": ("for (int i = 0; i < n; i++) r[i] = s[i] - omega * t[i];",
                            "for (int i = 0; i < n; i++) r[i] = s[i] + omega * t[i];",
                            lambda o: tbs.test_bicgstab_step_orthogonality(o)),
    "bicgstab_alpha_not_shadow": ("const double rv = dot(n, rh, v);", "const double rv = dot(n, r, v);",
                                  lambda o: tbs.test_bicgstab_step_orthogonality(o)),
    "bicgstab_p_drops_v": ("p[i] = r[i] + beta * (p[i] - omega * v[i]);", "p[i] = r[i] + beta * p[i];",
                           lambda o: tbs.test_bicgstab_alphas_equal_bicg(o)),
    "bicgstab_beta_inverted": ("const double beta = (rho / rho_prev) * (alpha / omega);",
                               "const double beta = (rho / rho_prev) * (omega / alpha);",
                               lambda o: tbs.test_bicgstab_alphas_equal_bicg(o)),
    "jacobi_divides_by_row_sum": ("for (int i = 0; i < n; i++) x[i] += r[i] / A[(long)i * lda + i];",
                                  "for (int i = 0; i < n; i++) x[i] += r[i] / A[(long)i * lda + i + 1];",
                                  lambda o: tja.test_jacobi_diagonal_one_update(o)),
    "jacobi_update_sign": ("for (int i = 0; i < n; i++) x[i] += r[i] / A[(long)i * lda + i];",
                           "for (int i = 0; i < n; i++) x[i] -= r[i] / A[(long)i * lda + i];",
                           lambda o: tja.test_jacobi_matches_lapack(o, 40)),
    "jacobi_gauss_seidel_sweep": ("for (int i = 0; i < n; i++) x[i] += r[i] / A[(long)i * lda + i];",
                                  "for (int i = 0; i < n; i++) { x[i] += r[i] / A[(long)i * lda + i];"
                                  " for (int q = i + 1; q < n; q++) r[q] -= A[(long)q * lda + i] * r[i]"
                                  " / A[(long)i * lda + i]; }",
                                  lambda o: tja.test_jacobi_rate_is_spectral_radius(o)),
    "gs_backward_sweep": ("for (int i = 0; i < n; i++) {                    /* the sweep, in place */",
                          "for (int i = n - 1; i >= 0; i--) {                    /* the sweep, in place */",
                          lambda o: tgs.test_gs_lower_triangular_is_forward_substitution(o)),
    "gs_drops_upper_part": ("if (j != i) s -= a[j] * x[j];", "if (j < i) s -= a[j] * x[j];",
                            lambda o: tgs.test_gs_matches_lapack(o, 40)),
    "gs_rhs_perturbed": ("            double s = b[i];\n", "            double s = b[i] * (1.0 + 1e-9);\n",
                         lambda o: tgs.test_gs_matches_lapack(o, 200)),
    "block_cg_alpha_transposed": ("const double a = al[c + j * s];", "const double a = al[j + c * s];",
                                  lambda o: tbc.test_block_cg_is_block_krylov_minimiser(o, 3, 5)),
    "block_cg_beta_transposed": ("for (int c = 0; c < s; c++) v += P[i + (long)c * n] * al[c + j * s];",
                                 "for (int c = 0; c < s; c++) v += P[i + (long)c * n] * al[j + c * s];",
                                 lambda o: tbc.test_block_cg_is_block_krylov_minimiser(o, 3, 5)),
    "block_cg_gamma_without_A": ("gram(n, s, P, Q, g);", "gram(n, s, P, P, g);",
                                 lambda o: tbc.test_block_cg_is_block_krylov_minimiser(o, 2, 3)),
    "block_gmres_rotation_sign": ("                    HB(r + 1, col) = 0.0;\n                    for (int q = 0; q < s; q++) {\n                        const double ga = GB(r, q), gb = GB(r + 1, q);\n                        GB(r, q) = cc * ga + ss * gb;\n                        GB(r + 1, q) = -ss * ga + cc * gb;",
                                  "                    HB(r + 1, col) = 0.0;\n                    for (int q = 0; q < s; q++) {\n                        const double ga = GB(r, q), gb = GB(r + 1, q);\n                        GB(r, q) = cc * ga + ss * gb;\n                        GB(r + 1, q) = ss * ga + cc * gb;",
                                  lambda o: tbg.test_block_gmres_is_block_krylov_minimiser(o, 3, 4)),
    "block_gmres_single_pass_basis_short": ("                    for (int q = 0; q < nb_idx; q++) {\n                        const double h = dot(n, V + (long)q * n, w);\n                        HB(q, col) += h;",
                                            "                    for (int q = 0; q < nb_idx - 1; q++) {\n                        const double h = dot(n, V + (long)q * n, w);\n                        HB(q, col) += h;",
                                            lambda o: tbg.test_block_gmres_is_block_krylov_minimiser(o, 3, 4)),
    "block_gmres_backsolve_index": ("for (int q = i + 1; q < k; q++) v -= HB(i, q) * y[q];",
                                    "for (int q = i + 1; q < k; q++) v -= HB(q, i) * y[q];",
                                    lambda o: tbg.test_block_gmres_is_block_krylov_minimiser(o, 2, 3)),
    "block_gmres_deflated_s_from_basis": ("GB(q, c) = dot(n, V + (long)q * n, R0 + (long)c * n);",
                                          "GB(q, c) = dot(n, V + (long)q * n, V + (long)c * n);",
                                          lambda o: tbg.test_deflated_block_gmres_rank_deficient_blocks_converge(o, 8)),
    "block_gmres_replacement_range": ("z[i] = 2.0 * ((double)(splitmix64_out(k) >> 11) * 0x1.0p-53) - 1.0;",
                                      "z[i] = 2.0 * ((double)(splitmix64_out(k) >> 11) * 0x1.0p-53) - 0.5;",
                                      lambda o: tbg.test_replacement_vectors_are_splitmix64(o)),
    "block_gmres_dependent_column_kept": ("dead[c] = !(nv > tol * before);", "dead[c] = !(nv > 0.0 * tol * before);",
                                          lambda o: tbg.test_deflated_block_gmres_minimises_over_kept_and_replacement_directions(o, 2)),
    # caught by the hand-derived worked examples (tests/golden)
    "ge_last_max_on_ties": ("if (a > best) { best = a; v = i; }", "if (a >= best) { best = a; v = i; }",
                            lambda o: tgo.test_lu_worked_example(o, "tie_")),
    "ge_swap_leaves_L": ("            for (int j = 0; j < n; j++) {\n                double t = W[(long)k * n + j];",
                         "            for (int j = k; j < n; j++) {\n                double t = W[(long)k * n + j];",
                         lambda o: tgo.test_lu_worked_example(o, "")),
    "cg_beta_inverted": ("double beta = rho_new / rho;", "double beta = rho / rho_new;",
                         lambda o: tgo.test_cg_worked_example(o)),
    "bicgstab_x_drops_omega_s": ("for (int i = 0; i < n; i++) x[i] += alpha * p[i] + omega * s[i];",
                                 "for (int i = 0; i < n; i++) x[i] += alpha * p[i];",
                                 lambda o: tgo.test_bicgstab_worked_example(o)),
    # the deflating block CG
    "bcgd_beta_sign": ("for (int i = 0; i < r; i++) be[i + j * r] = -dot(n, Q + (long)i * n, R + (long)j * n);",
                       "for (int i = 0; i < r; i++) be[i + j * r] = dot(n, Q + (long)i * n, R + (long)j * n);",
                       lambda o: tbd.test_full_rank_is_the_block_krylov_minimiser_and_oleary(o, 3, 5)),
    "bcgd_alpha_from_q": ("for (int i = 0; i < r; i++) al[i + j * r] = dot(n, P + (long)i * n, R + (long)j * n);",
                          "for (int i = 0; i < r; i++) al[i + j * r] = dot(n, Q + (long)i * n, R + (long)j * n);",
                          lambda o: tbd.test_s1_is_cg(o)),
    "bcgd_keeps_dependent": ("    const double tau = 1e-8;\n    const size_t nb",
                             "    const double tau = 0.0;\n    const size_t nb",
                             lambda o: tbd.test_rank_deficient_blocks_converge(o)),
    "chol_no_sqrt": ("double lkk = sqrt(akk);", "double lkk = akk;",
                     lambda o: tch.test_cholesky_worked_example(o)),
    "chol_update_reads_upper": ("W[(long)i * n + j] -= lik * W[(long)j * n + k];",
                                "W[(long)i * n + j] -= lik * W[(long)k * n + j];",
                                lambda o: tch.test_cholesky_matches_lapack_and_backward_error(o, 17)),
    "chol_back_solve_not_transposed": ("for (int j = i + 1; j < n; j++) s -= L[(long)j * n + i] * x[j];",
                                       "for (int j = i + 1; j < n; j++) s -= L[(long)i * n + j] * x[j];",
                                       lambda o: tch.test_cholesky_solve_matches_lapack(o, 33)),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new, pin = MUTATIONS[name]
    src = open(oracle_pkg.SOURCE).read()
    assert src.count(old) >= 1, "mutation site not found: " + name
    path = os.path.join(tmp_path, "mut.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new, 1))      # first occurrence (FP64 path)
    lib = oracle_pkg.compile_source(path, os.path.join(tmp_path, "libmut.so"))
    mutant = oracle_pkg.Oracle(lib)
    with pytest.raises(AssertionError):
        pin(mutant)
