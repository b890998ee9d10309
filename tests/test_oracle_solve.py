"""Pins for the plain multi-shift solve of the oracle (Eq. 2, Alg. 1, Alg. 3).

Each pin fixes the oracle against something other than itself: dense LAPACK
solves, a library triangular solve, a closed form, or an invariant.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1607_01477_gb300 import workloads as W
from conftest import EPS, backward_error


@pytest.mark.parametrize("m,n", [(1, 1), (7, 3), (33, 5), (64, 9)])
def test_solve_matches_dense_lapack(m, n):
    """Brute force: (U - s_j I) x_j = b_j solved densely by numpy.linalg.solve."""
    U, s, B = W.plain_problem(m, n, seed=100 + m)
    X = oracle.solve(U, s, B)
    for j in range(n):
        A = np.triu(U) - s[j] * np.eye(m)
        xd = np.linalg.solve(A, B[:, j])
        cond = np.linalg.cond(A)
        assert np.abs(X[:, j] - xd).max() <= 50 * m * EPS * cond * np.abs(xd).max()


def test_zero_shift_is_library_trsm():
    """Special case lambda = 0: the multi-shift solve is a plain TRSM (Sec. 2)."""
    U, _, B = W.plain_problem(48, 6, seed=7)
    X = oracle.solve(U, np.zeros(6, np.complex128), B)
    Xr = sla.solve_triangular(np.triu(U), B, lower=False)
    assert np.allclose(X, Xr, rtol=1e-11, atol=1e-11 * np.abs(Xr).max())


def test_diagonal_closed_form():
    """Diagonal U: x_j(i) = b_j(i) / (U(i,i) - s_j)."""
    g = W.rng(0, 11)
    m, n = 40, 7
    d = W.disk(g, m, 1.0)
    U = np.asfortranarray(np.diag(d))
    s = W.disk(g, n, 1.5)
    B = W.cn(g, (m, n))
    X = oracle.solve(U, s, B)
    Xc = B / (d[:, None] - s[None, :])
    assert np.abs(X - Xc).max() <= 4 * EPS * np.abs(Xc).max()


def test_backward_error_small():
    """Backward stability of back substitution (Sec. 2): eta_j <= c m eps."""
    U, s, B = W.plain_problem(256, 64, seed=1607014771)
    X = oracle.solve(U, s, B)
    eta = backward_error(U, s, X, B)
    assert eta.max() <= 256 * EPS


@pytest.mark.parametrize("m,nb", [(64, 16), (100, 32), (37, 8), (5, 8)])
def test_blocked_equals_unblocked(m, nb):
    """Alg. 3 (blocked, ragged top block) and Alg. 1 agree up to rounding (Sec. 2)."""
    U, s, B = W.plain_problem(m, 6, seed=3 * m + nb)
    X1 = oracle.solve(U, s, B)
    X3 = oracle.solve_blocked(U, s, B, nb)
    scale = np.abs(X1).max(axis=0)
    assert (np.abs(X1 - X3).max(axis=0) <= 1e-9 * scale).all()
    assert backward_error(U, s, X3, B).max() <= 64 * m * EPS


@pytest.mark.parametrize("m,n", [(1, 2), (30, 4), (64, 5)])
def test_conj_trans_matches_dense(m, n):
    """Lower (conjugate-transpose) case: (U^H - conj(s) I) x = b by forward substitution."""
    U, s, B = W.plain_problem(m, n, seed=900 + m)
    X = oracle.solve(U, s, B, conj_trans=True)
    for j in range(n):
        A = np.triu(U).conj().T - np.conj(s[j]) * np.eye(m)
        xd = np.linalg.solve(A, B[:, j])
        assert np.abs(X[:, j] - xd).max() <= 50 * m * EPS * np.linalg.cond(A) * np.abs(xd).max()


def test_trailing_zero_rhs_gives_trailing_zero_solution():
    """Footnote of Sec. 4: zeros at the bottom of b stay zeros in x."""
    U, s, B = W.plain_problem(30, 3, seed=5)
    B[20:, :] = 0
    X = oracle.solve(U, s, B)
    assert (X[20:, :] == 0).all()


def test_full_size_mixed_workload_sampled_columns():
    """The 8192 x 8192 workload with 2048 shifts (annulus diagonal, shifts in
    the disk of radius 0.4): the oracle's solution of 12 sampled columns has
    normwise backward error <= 8 m eps (Sec. 2: back substitution is backward
    stable), the bar the mixed-precision solve is held to after refinement."""
    U, s, B = W.mixed_problem()
    m, n = B.shape
    assert (m, n) == (8192, 2048)
    idx = np.array([0, 1, 511, 1024, 1500, 2047] + list(W.rng(0, 8192).choice(n, 6, replace=False)))
    Bs = np.asfortranarray(B[:, idx])
    X = oracle.solve(U, s[idx], Bs)
    assert np.isfinite(X).all()
    eta = backward_error(U, s[idx], X, Bs)
    assert eta.max() <= 8 * m * EPS
