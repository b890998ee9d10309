"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source: a transposed
operand, a wrong sign, a dropped conjugate, a dropped term or an off-by-one
rescale exponent. It builds the copy in a temporary directory as a separate
library, then runs one of the committed pins against it with the mutant in
place of the oracle. The pin must fail on the mutant (and it passes on the
oracle in its own test file). Nothing here touches the CUDA library.

Left out on purpose: a one-short k in the G >= Omega rescale (choose_k). It
leaves G in [Omega, 2 Omega), so the next G >= Omega test rescales once more
(k >= 1), and the last row, where G does not grow, always makes that test. The
outputs come out unchanged, so no pin on outputs can see this mutant.
"""
import importlib.util

import pytest

import oracle
import test_golden as t_golden
import test_oracle_adjoint as t_adjoint
import test_oracle_eig as t_eig
import test_oracle_gen as t_gen
import test_oracle_pseudo as t_pseudo
import test_oracle_pseudo1 as t_pseudo1
import test_oracle_safe as t_safe
import test_oracle_solve as t_solve
import test_oracle_trevc as t_trevc
import test_oracle_variants as t_variants

# (what the mistake is, text in msts_oracle.c, its replacement, occurrences,
#  pin module, pin function, pin arguments)
CASES = [
    ("back substitution reads U transposed",
     "b[r] = oz_sub(b[r], oz_mul(xi, AT(U, ldu, r, i)));",
     "b[r] = oz_sub(b[r], oz_mul(xi, AT(U, ldu, i, r)));", 1,
     t_solve, "test_solve_matches_dense_lapack", (33, 5)),
    ("pivot U(i,i) + lambda instead of U(i,i) - lambda",
     "b[i] = oz_div(b[i], oz_sub(AT(U, ldu, i, i), lambda));",
     "b[i] = oz_div(b[i], oz_add(AT(U, ldu, i, i), lambda));", 1,
     t_solve, "test_solve_matches_dense_lapack", (33, 5)),
    ("conjugate-transposed solve with the shift not conjugated",
     "oz piv = oz_sub(oz_conj(AT(U, ldu, i, i)), oz_conj(lambda));",
     "oz piv = oz_sub(oz_conj(AT(U, ldu, i, i)), lambda);", 1,
     t_solve, "test_conj_trans_matches_dense", (30, 4)),
    ("M >= Omega rescale one short (x(i) left at or above Omega)",
     "int kk = eM - (OR_OMEGA_EXP - 1);",
     "int kk = eM - OR_OMEGA_EXP;", 2,
     t_safe, "test_pow2_closed_form_bitwise", (1, 0)),
    ("block bound C_blk ||B(I1,j)|| dropped from G(j)",
     "G = G + P->cblk[b] * N;",
     "G = G + 0.0 * N;", 1,
     t_golden, "test_safe_rescale_exponent_fixture", ()),
    ("delta = 2 eps ||U||_inf",
     "double d = DBL_EPSILON * or_norm_inf_upper(m, U, ldu);",
     "double d = 2.0 * DBL_EPSILON * or_norm_inf_upper(m, U, ldu);", 1,
     t_safe, "test_exact_zero_pivot_uses_delta", ()),
    ("TREVC right-hand side +T(0:j-1,j) instead of -T(0:j-1,j)",
     "oz_make(-AT(T, ldt, r, j).re, -AT(T, ldt, r, j).im)",
     "AT(T, ldt, r, j)", 2,
     t_trevc, "test_two_by_two_closed_form", ()),
    ("Lanczos alpha with the wrong sign on the imaginary products",
     "a += vk[r].re * w[r].re + vk[r].im * w[r].im;",
     "a += vk[r].re * w[r].re - vk[r].im * w[r].im;", 1,
     t_pseudo, "test_exact_when_krylov_space_is_full", (16,)),
    ("Lanczos second solve with (T - zI)^T conjugated the wrong way",
     "trsv_shift_conj_trans(m, T, ldt, z[p], w);",
     "trsv_shift_conj_trans(m, T, ldt, oz_conj(z[p]), w);", 1,
     t_pseudo, "test_exact_when_krylov_space_is_full", (16,)),
    ("adjoint dU = -triu(Lambda X^T) (conjugate dropped)",
     "acc = oz_add(acc, oz_mul(AT(dB, lddb, r, j), oz_conj(X[c + j * m])));",
     "acc = oz_add(acc, oz_mul(AT(dB, lddb, r, j), X[c + j * m]));", 1,
     t_adjoint, "test_adjoint_matches_torch_autograd", (9, 3)),
    ("adjoint ds_j = x_j^T lambda_j (conjugate dropped)",
     "acc = oz_add(acc, oz_mul(oz_conj(X[r + j * m]), AT(dB, lddb, r, j)));",
     "acc = oz_add(acc, oz_mul(X[r + j * m], AT(dB, lddb, r, j)));", 1,
     t_adjoint, "test_adjoint_matches_torch_autograd", (9, 3)),
    ("generalized entries U + lambda V",
     "return oz_sub(AT(U, ldu, r, c), oz_mul(lambda, AT(V, ldv, r, c)));",
     "return oz_add(AT(U, ldu, r, c), oz_mul(lambda, AT(V, ldv, r, c)));", 1,
     t_gen, "test_plain_against_dense_solve", (33,)),
    ("back-transformation with Q transposed",
     "s = oz_add(s, oz_mul(AT(Q, ldq, i, k), AT(Z, ldz, k, j)));",
     "s = oz_add(s, oz_mul(AT(Q, ldq, k, i), AT(Z, ldz, k, j)));", 1,
     t_eig, "test_permutation_q_permutes_rows_exactly", ()),
    ("variant op(A) = A^H without the conjugate",
     "return op == 2 ? oz_conj(a) : a;",
     "return a;", 1,
     t_variants, "test_against_dense_solve", ("left", "upper", "C")),
    ("back substitution skips the last row of each AXPY",
     "for (int64_t r = 0; r < i; ++r)                            /* AXPY */",
     "for (int64_t r = 0; r + 1 < i; ++r)                            /* AXPY */", 1,
     t_solve, "test_solve_matches_dense_lapack", (33, 5)),
    ("rows below the block (I2) not rescaled when t < 1",
     "/* t < 1: rescale I0 and I2 */\n      for (int64_t r = 0; r < lo; ++r) x[r] = oz_ldexp(x[r], -kk);\n"
     "      for (int64_t r = hie; r < end; ++r) x[r] = oz_ldexp(x[r], -kk);",
     "/* t < 1: rescale I0 and I2 */\n      for (int64_t r = 0; r < lo; ++r) x[r] = oz_ldexp(x[r], -kk);", 1,
     t_safe, "test_pow2_closed_form_bitwise", (1, 8)),
    ("TREVC shortcut stops one row early",
     "int64_t end = shortcut ? (j < m ? j : m) : m;   /* active rows [0, end) */",
     "int64_t end = shortcut ? (j < m ? (j > 0 ? j - 1 : 0) : m) : m;", 1,
     t_trevc, "test_two_by_two_closed_form", ()),
    ("Lanczos vector divided by beta^2",
     "vn[r] = oz_scale(w[r], 1.0 / bn);",
     "vn[r] = oz_scale(w[r], 1.0 / (bn * bn));", 1,
     t_pseudo, "test_exact_when_krylov_space_is_full", (16,)),
    ("Sturm count with the wrong sign on b^2/d",
     "d = (a[i] - x) - b[i - 1] * b[i - 1] / d;",
     "d = (a[i] - x) + b[i - 1] * b[i - 1] / d;", 1,
     t_pseudo, "test_tridiag_max_matches_eigvalsh", (5,)),
    ("right-hand variant of A^H maps to A^H instead of conj(A)",
     "return trans == 0 ? 1 : (trans == 1 ? 0 : 3);",
     "return trans == 0 ? 1 : (trans == 1 ? 0 : 2);", 1,
     t_variants, "test_against_dense_solve", ("right", "upper", "C")),
    ("portrait grid margin a fifth instead of a quarter",
     "double h = 0.25 * (w > hgt ? w : hgt);",
     "double h = 0.2 * (w > hgt ? w : hgt);", 1,
     t_pseudo1, "test_portrait_grid_properties", ()),
    ("generalized block bound without |lambda| C_blk(V)",
     "G = G + (P->cblkU[b] + al * P->cblkV[b]) * N;",
     "G = G + P->cblkU[b] * N;", 1,
     t_golden, "test_safe_gsolve_rescale_exponent_fixture", ()),
    ("generalized column bound without |lambda| cin_V",
     "cnorm[i] = cnU[i] + al * cnV[i];",
     "cnorm[i] = cnU[i];", 1,
     t_golden, "test_safe_gsolve_rescale_exponent_fixture", ()),
    ("Higham's alternative vector scaled by 1/m instead of 2/(3m)",
     "double alt = 2.0 * norm1_vec(m, y) / (3.0 * (double)m);",
     "double alt = 2.0 * norm1_vec(m, y) / (2.0 * (double)m);", 1,
     t_pseudo1, "test_alternative_vector_estimate_when_it_wins", ()),
    ("safe lower variant reverses A transposed",
     "      U[r + c * (int64_t)mm] = rev ? op_entry(A, lda, op, m - 1 - r, m - 1 - c) : op_entry(A, lda, op, r, c);",
     "      U[r + c * (int64_t)mm] = rev ? op_entry(A, lda, op, m - 1 - c, m - 1 - r) : op_entry(A, lda, op, r, c);", 1,
     t_variants, "test_safe_pow2_closed_form_bitwise", ("left", "lower", "N", 8)),
    ("GeneralizedTriangEig eigenvalue S(j,j)/T(j,j) instead of T(j,j)/S(j,j)",
     "lam[j] = oz_div(AT(T, ldt, j, j), AT(S, lds, j, j));\n    for (int64_t r = 0; r < m; ++r)\n"
     "      AT(Z, ldz, r, j) = r < j ? oz_sub",
     "lam[j] = oz_div(AT(S, lds, j, j), AT(T, ldt, j, j));\n    for (int64_t r = 0; r < m; ++r)\n"
     "      AT(Z, ldz, r, j) = r < j ? oz_sub", 1,
     t_gen, "test_gtrevc_residual_and_directions", (60,)),
    ("1-norm estimator applies Q^T instead of Q^H",
     "s = oz_add(s, oz_mul(oz_conj(AT(Q, ldq, r, i)), x[r]));",
     "s = oz_add(s, oz_mul(AT(Q, ldq, r, i), x[r]));", 1,
     t_pseudo1, "test_estimate_is_attained_by_the_reported_vector", (17, True)),
]


def _mutant(tmp_path, old, new, count):
    """A second instance of the oracle's Python wrapper whose library is built
    from the mutated source in tmp_path."""
    src = open(oracle._SRC).read()
    assert src.count(old) == count, f"mutation site not found {count} times: {old}"
    path = tmp_path / "msts_oracle.c"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{tmp_path.name}", oracle.__file__)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._SRC = str(path)
    mod._LIB = str(tmp_path / "liboracle_mutant.so")
    mod._lib = None
    return mod


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pin_fails_on_planted_mistake(case, tmp_path):
    _, old, new, count, module, fn, args = case
    mut = _mutant(tmp_path, old, new, count)
    saved = module.oracle
    module.oracle = mut
    try:
        with pytest.raises(AssertionError):
            getattr(module, fn)(*args)
    finally:
        module.oracle = saved
