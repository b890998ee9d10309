"""Pins for the oracle's safe solves: Alg. 4 (SafeTrsv) and Alg. 5
(SafeMultiShiftTrsm), checked against closed forms and invariants."""
import numpy as np
import pytest

import oracle
from paper_1607_01477_gb300 import workloads as W
from conftest import EPS, backward_error

OMEGA = 2.0 ** 960


def bidiagonal_pow2(m, p, d_exp=-40):
    """U(i,i) = 2^d_exp, U(i,i+1) = -2^p, b = e_m: x(i) = 2^(-d_exp + (p - d_exp)(m-1-i))."""
    U = np.zeros((m, m), dtype=np.complex128, order="F")
    U[np.arange(m), np.arange(m)] = 2.0 ** d_exp
    U[np.arange(m - 1), np.arange(1, m)] = -(2.0 ** p)
    B = np.zeros((m, 1), dtype=np.complex128, order="F")
    B[m - 1, 0] = 1.0
    log2x = np.array([-d_exp + (p - d_exp) * (m - 1 - i) for i in range(m)])
    return U, B, log2x


@pytest.mark.parametrize("p", [0, 1, 3])
@pytest.mark.parametrize("nb", [0, 8, 5])
def test_pow2_closed_form_bitwise(p, nb):
    """Closed form with exact powers of two: x(i) * 2^e = 2^(40 + (p+40)(m-1-i)) exactly.
    The solution overflows double without scaling, so both the M >= Omega and the
    G >= Omega branches of Alg. 4 / Alg. 5 are taken; every value is a power of
    two, so the check is bitwise."""
    m = 32
    U, B, log2x = bidiagonal_pow2(m, p)
    s = np.zeros(1, dtype=np.complex128)
    if nb == 0:
        X, e = oracle.safe_trsv_unblocked(U, s, B)
    else:
        X, e = oracle.safe_solve(U, s, B, nb)
    assert e[0] > 0 and e[0] >= log2x.max() - 960
    expect = np.array([np.ldexp(1.0, int(k) - int(e[0])) for k in log2x])
    assert np.array_equal(X[:, 0].real, expect)
    assert (X[:, 0].imag == 0).all()
    assert np.abs(X).max() < OMEGA


def test_safe_equals_plain_when_no_bound_fires():
    """Sec. 3: if the bounds stay below Omega the safe solve is the plain one with
    s = 1; the blocked safe solve then repeats Alg. 3's arithmetic bit for bit."""
    U, s, B = W.plain_problem(100, 12, seed=21)
    Xs, e = oracle.safe_solve(U, s, B, 16)
    Xp = oracle.solve_blocked(U, s, B, 16)
    assert (e == 0).all()
    assert np.array_equal(Xs, Xp)


def test_safe_scaled_solution_matches_plain_when_representable():
    """x_j / s_j equals the plain solution whenever that one is finite: growth that
    exceeds Omega = 2^960 but stays below DBL_MAX."""
    m = 24
    U, B, _ = bidiagonal_pow2(m, 2, d_exp=-40)
    g = W.rng(0, 5)
    U[np.triu_indices(m, 2)] = 1e-3 * W.cn(g, (m, m))[np.triu_indices(m, 2)]
    s = np.array([0.25 + 0.1j], dtype=np.complex128) * 0  # exact shift 0
    Xp = oracle.solve(U, s, B)
    assert np.isfinite(Xp).all() and np.abs(Xp).max() > OMEGA
    for nb in (0, 6, 8):
        X, e = (oracle.safe_trsv_unblocked(U, s, B) if nb == 0 else oracle.safe_solve(U, s, B, nb))
        assert e[0] > 0
        Xr = np.ldexp(X.real, int(e[0])) + 1j * np.ldexp(X.imag, int(e[0]))
        assert np.abs(Xr - Xp).max() <= 1e-12 * np.abs(Xp).max()


@pytest.mark.parametrize("nb", [8, 32])
def test_invariants_on_hard_trevc_like_input(nb):
    """s_j in [0,1], finite x below Omega, and a small scaled residual
    ||(U - l I) x - s b|| / (||U - l I|| ||x|| + s ||b||) (Sec. 3)."""
    m = 256
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    lam = np.diag(T).copy()
    g = W.rng(0, 9)
    B = W.cn(g, (m, 20))
    shifts = lam[g.permutation(m)[:20]] + 1e-9
    X, e = oracle.safe_solve(T, shifts, B, nb)
    assert (e >= 0).all() and e.max() > 0
    assert np.isfinite(X).all() and np.abs(X).max() < OMEGA
    sc = np.ldexp(1.0, -e.astype(np.int64))
    eta = backward_error(T, shifts, X, B, scales=sc)
    assert eta.max() <= 64 * m * EPS


def test_blocked_and_unblocked_safe_agree_up_to_scale():
    """Both safe variants solve the same systems; x/s agree wherever s is not tiny."""
    T = W.trevc_problem(64, seed=3, offdiag_scale=3.0)
    g = W.rng(0, 4)
    B = W.cn(g, (64, 10))
    shifts = W.disk(g, 10, 1.0)
    X1, e1 = oracle.safe_trsv_unblocked(T, shifts, B)
    X5, e5 = oracle.safe_solve(T, shifts, B, 16)
    for j in range(10):
        a = X1[:, j] * 2.0 ** (e5[j] - e1[j]) if e5[j] >= e1[j] else X1[:, j]
        b = X5[:, j] if e5[j] >= e1[j] else X5[:, j] * 2.0 ** (e1[j] - e5[j])
        assert np.abs(a - b).max() <= 1e-8 * np.abs(b).max()


def test_exact_zero_pivot_uses_delta():
    """U(i,i) = lambda exactly: the pivot is replaced by delta = eps ||U||_inf (Sec. 3)
    and the solve stays finite with a small scaled residual."""
    U, s, B = W.plain_problem(40, 3, seed=8)
    s[1] = U[17, 17]
    X, e = oracle.safe_solve(U, s, B, 8)
    assert np.isfinite(X).all()
    sc = np.ldexp(1.0, -e.astype(np.int64))
    assert backward_error(U, s, X, B, scales=sc).max() <= 64 * 40 * EPS
    assert oracle.delta(U) == pytest.approx(EPS * np.abs(np.triu(U)).sum(axis=1).max(), rel=1e-12, abs=0)


def test_zero_rhs_and_empty():
    U, s, B = W.plain_problem(20, 3, seed=1)
    B[:] = 0
    X, e = oracle.safe_solve(U, s, B, 8)
    assert (X == 0).all() and (e == 0).all()
