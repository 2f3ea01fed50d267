"""The oracle's pins catch plausible mistakes planted in the oracle.

Each case copies the oracle's C source, plants one mistake of the kind a
reader checking it against the paper could miss (a wrong sign, a dropped
term, a wrong index, a transposed operand, an off-by-one), builds the copy and
runs, in a child process that loads that build, the pins that must catch it:
they must fail.  The unmodified source, built and run the same way, passes
every one of those pins, so a failure is the planted mistake's doing.  The
oracle's own source and library are not touched.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mgpbd_oracle.c")
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-shared", "-fPIC"]
PINS = "tests/test_oracle_pins.py::"
ARAP = "tests/test_oracle_arap.py::"
NK = "tests/test_oracle_nearkernel.py::"

# (name, passage, original text, planted text, pins that must fail)
MUTANTS = [
    ("distance_gradient_sign", "Eq. 3, distance gradient n = (x_a - x_b)/|x_a - x_b|",
     "if (len > 0.0) { n[0] = d0 / len; n[1] = d1 / len; n[2] = d2 / len; }",
     "if (len > 0.0) { n[0] = -d0 / len; n[1] = -d1 / len; n[2] = -d2 / len; }",
     [PINS + "test_gradients_match_finite_differences[0]"]),
    ("volume_without_sixth", "Eq. 3, tetrahedron volume det/6",
     "double V = fma(e1[2], c23[2], fma(e1[1], c23[1], e1[0] * c23[0])) / 6.0;",
     "double V = fma(e1[2], c23[2], fma(e1[1], c23[1], e1[0] * c23[0]));",
     [PINS + "test_constraint_closed_forms"]),
    ("volume_gradient_transposed_cross", "Eq. 3, volume gradient (x2-x0) x (x3-x0)/6",
     "cross(e2, e3, c23); cross(e3, e1, c31);", "cross(e3, e2, c23); cross(e3, e1, c31);",
     [PINS + "test_gradients_match_finite_differences[1]"]),
    ("rhs_sign_of_compliance_term", "Eq. 3, b = -C - alpha~ lambda",
     "o->b[j] = (-o->C[j]) - t;", "o->b[j] = (-o->C[j]) + t;",
     [PINS + "test_single_constraint_stays_at_the_compliant_solution"]),
    ("diagonal_without_compliance", "Eq. 3, A = J M^-1 J^T + alpha~",
     "o->A.val[e] = acc + o->alpha_t[i];", "o->A.val[e] = acc;",
     [PINS + "test_A_equals_dense_J_Minv_JT_plus_alpha[0]"]),
    ("off_diagonal_wrong_vertex_weight", "Sec. 4.2, A_ij sums w_v over shared vertices",
     "acc = fma(o->w[vv[si]], gdot(gi[si], gj), acc);",
     "acc = fma(o->w[vv[0]], gdot(gi[si], gj), acc);",
     [PINS + "test_A_equals_dense_J_Minv_JT_plus_alpha[1]"]),
    ("pattern_diagonal_not_last", "Sec. 4.2, off-diagonals first, diagonal last",
     "    col[base + cnt] = i; /* diagonal last */",
     "    col[base + cnt] = tmp[0] >= 0 && cnt ? tmp[0] : i; /* diagonal last */",
     [PINS + "test_pattern_brute_force[0]"]),
    ("strength_without_sqrt", "Sec. 4.1, strength threshold theta sqrt(|A_ii A_jj|)",
     "double thr = theta * sqrt(prod);", "double thr = theta * prod;",
     [PINS + "test_strength_hand_example"]),
    ("strength_equality_weak", "Sec. 4.1, weak only below the threshold",
     "S[k] = fabs(A->val[k]) >= thr;", "S[k] = fabs(A->val[k]) > thr;",
     [PINS + "test_strength_hand_example"]),
    ("aggregation_weakest_connection", "Sec. 4.1, leftover rows join the most strongly coupled aggregate",
     "double s = fabs(A->val[k]);", "double s = 1.0 / fabs(A->val[k]);",
     [PINS + "test_aggregation_brute_force[0.1-0]"]),
    ("aggregation_distance_one_roots", "Sec. 4.1, roots independent at strength distance 2",
     "if (S[k2]) blocked[A->col[k2]] = 1;", "if (S[k2] && 0) blocked[A->col[k2]] = 1;",
     [PINS + "test_aggregation_brute_force[0.1-0]"]),
    ("injection_not_normalised", "Sec. 4.1, P_i = B_i / |B_a|",
     "L->P[i] = nrm > 0.0 ? L->B[i] / nrm : 1.0 / sqrt((double)sz);",
     "L->P[i] = nrm > 0.0 ? L->B[i] : 1.0 / sqrt((double)sz);",
     [PINS + "test_prolongator_and_galerkin[c8]"]),
    ("galerkin_wrong_index", "Eq. 6, P_i A_ij P_j",
     "acc[b] = fma(t, L->P[j], acc[b]);", "acc[b] = fma(t, L->P[i], acc[b]);",
     [PINS + "test_prolongator_and_galerkin[c8]"]),
    ("galerkin_mirror_from_itself", "Eq. 6, symmetric coarse operator",
     "if (b < a) Ac->val[k] = Ac->val[find_col(Ac, b, a)];",
     "if (b < a) Ac->val[k] = Ac->val[find_col(Ac, a, b)];",
     [PINS + "test_prolongator_and_galerkin[c8]"]),
    ("near_kernel_sweep_sign", "Sec. 4.3, weighted Jacobi on A x = 0",
     "B[i] = fma(-p->nk_omega, s[i] / diag_of(A, i), B[i]);",
     "B[i] = fma(p->nk_omega, s[i] / diag_of(A, i), B[i]);",
     [PINS + "test_near_kernel_is_weighted_jacobi_on_homogeneous_system"]),
    ("near_kernel_start_unscaled", "Sec. 4.3, random start scaled by max|A_ij|",
     "for (int i = 0; i < n; ++i) B[i] = u01(h64(hkey(seed, 0, i))) * amax;",
     "for (int i = 0; i < n; ++i) B[i] = u01(h64(hkey(seed, 0, i)));",
     [PINS + "test_near_kernel_is_weighted_jacobi_on_homogeneous_system"]),
    ("six_vectors_R_not_accumulated", "Sec. 4.3, k vectors: QR of each aggregate",
     "R[d * k + c] = pass ? R[d * k + c] + r : r;", "R[d * k + c] = r;",
     [NK + "test_qr_of_each_aggregate[c8]"]),
    ("six_vectors_prolong_first_column", "Sec. 4.3, k vectors: k coarse unknowns per aggregate",
     "L->x[i] = fma(L->P[(size_t)i * k + c], Lc->x[L->agg[i] * k + c], L->x[i]);",
     "L->x[i] = fma(L->P[(size_t)i * k + c], Lc->x[L->agg[i] * k], L->x[i]);",
     [NK + "test_vcycle_symmetric_with_k_columns[c8]"]),
    ("power_method_without_diagonal", "Sec. 4.5, lambda_max of D^-1 A",
     "for (int i = 0; i < n; ++i) z[i] = z[i] / diag_of(A, i);",
     "for (int i = 0; i < n; ++i) z[i] = z[i];",
     [PINS + "test_power_method_omega[c8]"]),
    ("omega_without_safety_factor", "Sec. 4.5, omega = 2/(lambda_max + lambda_min)",
     "L->omega = 2.0 / (o->p.power_safety * L->lmax + o->p.lambda_min_est);",
     "L->omega = 2.0 / (L->lmax + o->p.lambda_min_est);",
     [PINS + "test_power_method_omega[c8]"]),
    ("jacobi_residual_sign", "Sec. 4.5, weighted Jacobi smoothing",
     "x[i] = fma(L->omega, (b[i] - t[i]) / diag_of(&L->A, i), x[i]);",
     "x[i] = fma(L->omega, (t[i] - b[i]) / diag_of(&L->A, i), x[i]);",
     [PINS + "test_pcg_matches_dense_cholesky[c8-0]"]),
    ("colouring_skips_a_neighbour", "Sec. 4.5, multicolour ordering",
     "for (int64_t k = A->ptr[u]; k < A->ptr[u + 1] - 1; ++k) {\n      int c = color[A->col[k]];",
     "for (int64_t k = A->ptr[u]; k < A->ptr[u + 1] - 2; ++k) {\n      int c = color[A->col[k]];",
     [PINS + "test_colouring_is_greedy_by_priority[0]"]),
    ("gauss_seidel_post_sweep_forward", "Sec. 4.4, symmetric pre- and post-smoothing",
     "else for (int c = L->n_colors - 1; c >= 0; --c) gs_colour(L, x, b, c);",
     "else for (int c = 0; c < L->n_colors; ++c) gs_colour(L, x, b, c);",
     [PINS + "test_vcycle_is_symmetric[c8-1]"]),
    ("chebyshev_recurrence_sign", "Sec. 4.5, Chebyshev smoother",
     "double rho2 = 1.0 / (2.0 * sigma - rho);", "double rho2 = 1.0 / (2.0 * sigma + rho);",
     [PINS + "test_chebyshev_matches_the_chebyshev_polynomial"]),
    ("restriction_of_rhs_not_residual", "Sec. 4.4, V-cycle restricts the residual",
     "acc = fma(L->P[(size_t)i * k + c], L->r[i], acc);",
     "acc = fma(L->P[(size_t)i * k + c], L->b[i], acc);",
     [PINS + "test_vcycle_is_symmetric[c8-0]"]),
    ("prolongation_sign", "Sec. 4.4, V-cycle adds the coarse correction",
     "L->x[i] = fma(L->P[(size_t)i * k + c], Lc->x[L->agg[i] * k + c], L->x[i]);",
     "L->x[i] = fma(-L->P[(size_t)i * k + c], Lc->x[L->agg[i] * k + c], L->x[i]);",
     [PINS + "test_pcg_matches_dense_cholesky[c8-0]"]),
    ("cholesky_wrong_index", "coarsest level: dense Cholesky",
     "for (int k = 0; k < j; ++k) s = fma(-Lm[(size_t)i * n + k], Lm[(size_t)j * n + k], s);",
     "for (int k = 0; k < j; ++k) s = fma(-Lm[(size_t)i * n + k], Lm[(size_t)i * n + k], s);",
     [PINS + "test_one_level_hierarchy_converges_in_one_iteration"]),
    ("back_substitution_wrong_index", "coarsest level: triangular solves",
     "for (int k = i + 1; k < n; ++k) s = fma(-Lm[(size_t)k * n + i], x[k], s);",
     "for (int k = i + 1; k < n; ++k) s = fma(-Lm[(size_t)i * n + k], x[k], s);",
     [PINS + "test_one_level_hierarchy_converges_in_one_iteration"]),
    ("pcg_beta_inverted", "Sec. 4.4, PCG beta = r'z' / r.z",
     "double be = rz2 / rz;", "double be = rz / rz2;",
     [PINS + "test_pcg_matches_dense_cholesky[c8-0]"]),
    ("position_update_wrong_vertex", "Eq. 5, dx_v = w_v sum_j grad_v C_j dlambda_j",
     "      row_grad(o, j, s, g);\n      for (int k = 0; k < 3; ++k) acc[k] = fma(g[k], o->dl[j], acc[k]);",
     "      row_grad(o, j, 0, g);\n      for (int k = 0; k < 3; ++k) acc[k] = fma(g[k], o->dl[j], acc[k]);",
     [PINS + "test_single_constraint_reduces_to_xpbd_update[1.0]"]),
    ("lambda_not_accumulated", "Alg. 1, lambda += dlambda",
     "o->lambda[j] = o->lambda[j] + o->dl[j];", "o->lambda[j] = o->dl[j];",
     [PINS + "test_single_constraint_stays_at_the_compliant_solution"]),
    ("relaxation_ignored", "Sec. 4, x += omega_x dx",
     "for (int64_t q = 0; q < n3; ++q) o->x[q] = fma(om, o->dx[q], o->x[q]);",
     "for (int64_t q = 0; q < n3; ++q) o->x[q] = o->x[q] + o->dx[q];",
     [PINS + "test_single_constraint_reduces_to_xpbd_update[0.25]"]),
    ("backtracking_never_halves", "Sec. 4, omega halves while the residual grows",
     "om = om * 0.5;", "om = om * 1.0;",
     [PINS + "test_backtracking_never_accepts_a_growing_residual_when_a_halving_helps"]),
    ("explicit_euler_position", "Alg. 1, semi-implicit Euler",
     "double t2 = o->p.dt * vel[k];", "double t2 = o->p.dt * (vel[k] - t);",
     [PINS + "test_free_fall_without_constraints"]),
    ("gravity_moves_pinned_vertices", "Alg. 1, pinned vertices (w = 0) stay",
     "if (o->w[v] == 0.0) { vel[0] = vel[1] = vel[2] = 0.0; continue; }",
     "if (o->w[v] == 0.0 && 0) { vel[0] = vel[1] = vel[2] = 0.0; continue; }",
     [PINS + "test_free_fall_without_constraints"]),
    ("velocity_sign", "Alg. 1, v = (x - x_old)/dt",
     "o->v[q] = (o->x[q] - o->xold[q]) / o->p.dt;", "o->v[q] = (o->xold[q] - o->x[q]) / o->p.dt;",
     [PINS + "test_free_fall_without_constraints"]),
    ("xpbd_local_step_sign", "Eq. 4, dlambda_j = b_j / A_jj",
     "for (int j = 0; j < o->m; ++j) o->dl[j] = o->b[j] / diag_of(&o->A, j);",
     "for (int j = 0; j < o->m; ++j) o->dl[j] = -o->b[j] / diag_of(&o->A, j);",
     [PINS + "test_xpbd_step_is_the_diagonal_solve_and_stalls_where_mgpcg_does_not"]),
    ("arap_polar_inverse_not_inverse_transpose", "Sec. 5.3, polar rotation R",
     "R[a][k] = 0.5 * (R[a][k] + dual[k][a] / det);",
     "R[a][k] = 0.5 * (R[a][k] + dual[a][k] / det);",
     [ARAP + "test_polar_factor_closed_form"]),
    ("arap_gradient_without_two", "Sec. 5.3, dC/dF = 2 (F - R)",
     "g[3 * (k + 1) + a] = 2.0 * t;", "g[3 * (k + 1) + a] = t;",
     [ARAP + "test_gradient_matches_finite_differences"]),
    ("six_vectors_one_seed", "Sec. 4.3, k near-kernel vectors from independent starts",
     "near_kernel_one(A, p, p->seed_nk + (uint64_t)c, v);", "near_kernel_one(A, p, p->seed_nk, v);",
     [NK + "test_near_kernel_columns_are_the_single_vector_procedure"]),
    ("node_norm_one_norm", "Sec. 4.3, k vectors: node strength from k x k block norms",
     "        *c = fma(v, v, *c);", "        *c = *c + fabs(v);",
     [NK + "test_coarse_levels_aggregate_whole_nodes"]),
    ("node_norm_without_sqrt", "Sec. 4.3, k vectors: Frobenius norm of a block",
     "for (int t = 0; t <= cnt; ++t) N->val[base + t] = sqrt(N->val[base + t]);",
     "for (int t = 0; t <= cnt; ++t) N->val[base + t] = N->val[base + t];",
     [NK + "test_coarse_levels_aggregate_whole_nodes"]),
    ("galerkin_k_wrong_column", "Eq. 6 with k columns, P_ip A_ij P_jq",
     "*cell = fma(t, L->P[(size_t)j * k + qq], *cell);",
     "*cell = fma(t, L->P[(size_t)j * k + p], *cell);",
     [NK + "test_galerkin_with_k_columns[c8]"]),
    ("galerkin_k_dead_diagonal_zero", "Sec. 4.3, k vectors: dropped columns keep the coarse matrix SPD",
     "if (L->pdead[r]) Ac->val[Ac->ptr[r + 1] - 1] = 1.0;",
     "if (L->pdead[r]) Ac->val[Ac->ptr[r + 1] - 1] = 0.0;",
     [NK + "test_galerkin_with_k_columns[c8]"]),
    ("qr_without_drop_tolerance", "Sec. 4.3, k vectors: numerically dependent columns dropped",
     "int live = nv > 0.0 && nrm > ORC_QR_DROP * sqrt(nb);", "int live = nv > 0.0;",
     [NK + "test_qr_of_each_aggregate[c8]"]),
    ("chebyshev_start_unscaled", "Sec. 4.5, Chebyshev smoother's first step r/theta",
     "d[i] = r[i] / theta;", "d[i] = r[i];",
     [PINS + "test_chebyshev_matches_the_chebyshev_polynomial"]),
    ("backtracking_stops_on_growth", "Sec. 4, omega halves while the residual grows",
     "if (nb < info->bnorm || t == o->p.backtrack) break;",
     "if (nb > info->bnorm || t == o->p.backtrack) break;",
     [PINS + "test_backtracking_never_accepts_a_growing_residual_when_a_halving_helps"]),
    ("position_update_without_inverse_mass", "Eq. 5, dx = M^-1 grad C^T dlambda",
     "o->dx[3 * (int64_t)v + k] = o->w[v] * acc[k];", "o->dx[3 * (int64_t)v + k] = acc[k];",
     [PINS + "test_single_constraint_reduces_to_xpbd_update[1.0]"]),
    ("cholesky_without_pivot_check", "coarsest level: a zero pivot is singular",
     "if (!(d > 0.0)) return ORC_E_SINGULAR;", "if (0) return ORC_E_SINGULAR;",
     [PINS + "test_singular_system_is_reported"]),
    ("arap_rest_inverse_transposed", "Sec. 5.3, F = Ds Dm^-1",
     "for (int k = 0; k < 3; ++k) B[3 * r + k] = det != 0.0 ? c[r][k] / det : 0.0;",
     "for (int k = 0; k < 3; ++k) B[3 * r + k] = det != 0.0 ? c[k][r] / det : 0.0;",
     [ARAP + "test_polar_factor_on_a_skewed_rest_shape"]),
    ("arap_singular_deformation_unhandled", "Sec. 5.3, no polar factor for a singular F",
     "  if (detF == 0.0) {", "  if (0) {",
     [ARAP + "test_singular_and_reflected_deformations"]),
    ("jacobi_without_weight", "Sec. 4.5, omega-weighted Jacobi",
     "x[i] = fma(L->omega, (b[i] - t[i]) / diag_of(&L->A, i), x[i]);",
     "x[i] = x[i] + (b[i] - t[i]) / diag_of(&L->A, i);",
     [PINS + "test_chebyshev_degree_one_is_optimal_weighted_jacobi"]),
    ("pcg_alpha_wrong_denominator", "Sec. 4.4, PCG alpha = r.z / p.Ap",
     "double al = rz / pq;", "double al = rz / rr;",
     [PINS + "test_one_level_hierarchy_converges_in_one_iteration"]),
    ("true_residual_sign", "Sec. 4.4, true residual b - A dlambda",
     "for (int i = 0; i < n; ++i) q[i] = b[i] - q[i];",
     "for (int i = 0; i < n; ++i) q[i] = b[i] + q[i];",
     [PINS + "test_pcg_matches_dense_cholesky[c8-0]"]),
    ("lambda_not_reset_per_frame", "Alg. 1, lambda = 0 at the start of a time step",
     "  memset(o->lambda, 0, sizeof(double) * (size_t)o->m);\n}", "}",
     [PINS + "test_single_constraint_stays_at_the_compliant_solution"]),
    ("strength_with_signed_scaled_diagonal", "Sec. 4.1, strength uses |A_ii|",
     "double aii = fabs(diag_of(A, i));", "double aii = diag_of(A, i) * 0.5;",
     [PINS + "test_aggregation_brute_force[0.1-0]"]),
    ("six_vectors_restrict_first_column", "Sec. 4.3, k vectors: restriction by every column of P",
     "acc = fma(L->P[(size_t)i * k + c], L->r[i], acc);\n      }\n      Lc->b[a * k + c] = acc;",
     "acc = fma(L->P[(size_t)i * k], L->r[i], acc);\n      }\n      Lc->b[a * k + c] = acc;",
     [NK + "test_pcg_with_k_columns_matches_dense_cholesky[c8]"]),
    ("splitmix_shift", "counter-based generator (SplitMix64 finaliser)",
     "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;",
     [PINS + "test_splitmix64_reference_values"]),
]


def _build_and_run(workdir, name, source, pins):
    d = os.path.join(workdir, name)
    os.makedirs(d, exist_ok=True)
    c, so = os.path.join(d, "oracle.c"), os.path.join(d, "liborc.so")
    with open(c, "w") as f:
        f.write(source)
    subprocess.run(["gcc", *CFLAGS, c, "-o", so, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, MGPBD_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        *pins], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(SRC).read()
    work = str(tmp_path_factory.mktemp("mutants"))
    jobs = {"unmodified": (src, sorted({p for m in MUTANTS for p in m[4]}))}
    for name, _, old, new, pins in MUTANTS:
        assert src.count(old) == 1, f"{name}: the original text must occur exactly once"
        jobs[name] = (src.replace(old, new), pins)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {k: ex.submit(_build_and_run, work, k, s, p) for k, (s, p) in jobs.items()}
        return {k: f.result() for k, f in futs.items()}


def test_unmodified_source_passes_every_pin_used(outcomes):
    rc, out = outcomes["unmodified"]
    assert rc == 0, out


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, name):
    rc, out = outcomes[name]
    # 1: pytest ran the pins and at least one failed (not a crash or a usage error)
    assert rc == 1, f"{name} survived or did not run (exit {rc}):\n{out}"
