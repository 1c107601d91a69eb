"""The pins are strong enough: each test plants one plausible mistake in a copy of
the oracle's C source (on the CPU), loads the mutant and checks that at least one
pin fails. The real oracle is restored afterwards."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "fe_oracle.c")

MUTANTS = {
    "shear_modulus_doubled": ("for (int i = 3; i < 6; ++i) D[i][i] = mu;", "for (int i = 3; i < 6; ++i) D[i][i] = 2.0 * mu;"),
    "quadrature_weight": ("double w = det / 24.0;", "double w = det / 6.0;"),
    "edge_shape_factor": ("dN[4 + q][k] = 4.0 * (L[b] * dL[a][k] + L[a] * dL[b][k]);",
                          "dN[4 + q][k] = 2.0 * (L[b] * dL[a][k] + L[a] * dL[b][k]);"),
    "corner_shape_sign": ("dN[a][k] = (4.0 * L[a] - 1.0) * dL[a][k];", "dN[a][k] = (4.0 * L[a] + 1.0) * dL[a][k];"),
    "shear_row_swapped": ("B[4][c + 0] = g[2]; B[4][c + 2] = g[0];   /* gamma_xz */",
                          "B[4][c + 0] = g[0]; B[4][c + 2] = g[2];   /* gamma_xz */"),
    "lame_lambda": ("double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));",
                    "double lam = E * nu / ((1.0 + nu) * (1.0 - nu));"),
    "jacobian_transposed": ("for (int k = 0; k < 3; ++k) J[i][k] += xe[3 * n + i] * dN[n][k];",
                            "for (int k = 0; k < 3; ++k) J[k][i] += xe[3 * n + i] * dN[n][k];"),
    "bc_diagonal_zero": ("if (!fi || !fj) vals[9 * b + 3 * i + j] = (n == m && i == j) ? 1.0 : 0.0;",
                         "if (!fi || !fj) vals[9 * b + 3 * i + j] = 0.0;"),
    "bc_columns_kept": ("if (!fi || !fj) vals[9 * b + 3 * i + j] = (n == m && i == j) ? 1.0 : 0.0;",
                        "if (!fi) vals[9 * b + 3 * i + j] = (n == m && i == j) ? 1.0 : 0.0;"),
    "pcg_residual_sign": ("          r[k] -= alpha * q[k];\n        }\n      }\n    apply_blocks(N, R, Minv, r, z);",
                          "          r[k] += alpha * q[k];\n        }\n      }\n    apply_blocks(N, R, Minv, r, z);"),
    "adjoint_sign": ("    g[e] = -acc;", "    g[e] = acc;"),
    "aggregate_stragglers_to_last": ("    agg[n] = first[best];", "    agg[n] = (int32_t)(count - 1);"),
    "galerkin_column_aggregate": ("        const int32_t B = agg[b];", "        const int32_t B = agg[a];"),
    "inner_literal_n_minus_1": ("  for (int step = 0; step < n_steps; ++step) {\n    dots_f32(N, R, eb, eb, en);",
                                "  for (int step = 0; step < n_steps - 1; ++step) {\n    dots_f32(N, R, eb, eb, en);"),
    "inner_ratio_unsquared": ("if (active[c] && rbn[c] > 0.0 && en[c] / rbn[c] > worst) worst = en[c] / rbn[c];",
                              "if (active[c] && rbn[c] > 0.0 && sqrt(en[c] / rbn[c]) > worst) worst = sqrt(en[c] / rbn[c]);"),
    "inner_max_over_all_cases": ("if (active[c] && rbn[c] > 0.0 && en[c] / rbn[c] > worst) worst = en[c] / rbn[c];",
                                 "if (rbn[c] > 0.0 && en[c] / rbn[c] > worst) worst = en[c] / rbn[c];"),
    "block_jacobi_transposed": ("for (int j = 0; j < 3; ++j) A[i][j] = vals[9 * b + 3 * i + j];",
                                "for (int j = 0; j < 3; ++j) A[i][j] = vals[9 * b + 3 * j + i] * (i == j ? 1.0 : 0.5);"),
}

PINS = [
    pins.test_element_rigid_body_modes_and_rank,
    pins.test_element_symmetric,
    pins.test_element_linear_energy_closed_form,
    pins.test_element_quadratic_energy_closed_form,
    pins.test_element_scaling_and_material_linearity,
    pins.test_constrained_spd_and_symmetric,
    pins.test_block_jacobi_inverts_diagonal_blocks,
    pins.test_linear_patch_test,
    pins.test_quadratic_patch_test,
    pins.test_oedometer_exact,
    pins.test_adjoint_gradient_matches_finite_differences,
    lambda: pins.test_aggregation_is_a_partition_into_connected_aggregates(pins.make_tet4_levels()),
    lambda: pins.test_galerkin_aggregation_matrix_is_the_triple_product(pins.make_tet4_levels()),
]


def _box8():
    m = pins.mg.plain_box()
    return m, oracle.assemble(m), pins.mg.plain_box_rhs(m)


# pins of the inner loop of Algorithm 1(b)
PINS += [lambda: pins.test_fcg_inner_loop_runs_n0_steps_when_eps_is_zero(_box8()),
         lambda: pins.test_fcg_inner_stop_rule_is_on_the_squared_ratio(_box8()),
         lambda: pins.test_fcg_inner_stop_ignores_converged_cases(_box8())]


def _solver_pin():
    m = pins.mg.plain_box(n=3)
    K = oracle.assemble(m)
    f = pins.mg.plain_box_rhs(m)
    ud = oracle.direct_solve(K, f)
    u, it, rel = oracle.pcg(K, f, tol=1e-10, maxit=2000)
    assert rel[0] <= 1e-9
    assert np.linalg.norm(u - ud) <= 1e-6 * np.linalg.norm(ud)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib_path = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC", str(mut), "-o",
                    str(lib_path), "-lm"], check=True)
    saved = oracle._load()
    oracle._lib = oracle.configure(ctypes.CDLL(str(lib_path)))
    failed = []
    try:
        for pin in PINS + [_solver_pin]:
            try:
                pin()
            except Exception as exc:  # a pin failed (assertion or an error raised by the mutant)
                failed.append((pin.__name__, type(exc).__name__))
    finally:
        oracle._lib = saved
    assert failed, f"no pin caught mutant {name}"
