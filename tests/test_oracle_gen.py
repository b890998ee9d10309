"""Pins of the oracle's generalized multi-shift solves (appendix, Alg. 8-10):
(U - s_j V) x_j = b_j and GeneralizedTriangEig, against what the mathematics
fixes -- reductions to the standard solve, dense solves, closed forms, safe
invariants, and generalized eigen-residuals and directions."""
import numpy as np
import pytest
import scipy.linalg

import oracle
from paper_1607_01477_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def gen_pair(m, seed, vdiag=1.0):
    g = W.rng(0, seed)
    U = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(W.disk(g, m, 1.0)))
    V = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(vdiag + 0.2 * W.disk(g, m, 1.0)))
    return g, U, V


@pytest.mark.parametrize("m,n,nb", [(1, 1, 16), (40, 5, 16), (97, 9, 32), (130, 7, 64)])
def test_identity_v_is_the_standard_solve_bitwise(m, n, nb):
    U, s, B = W.plain_problem(m, n, seed=300 + m)
    I = np.asfortranarray(np.eye(m, dtype=np.complex128))
    assert np.array_equal(oracle.gsolve(U, I, s, B), oracle.solve(U, s, B))
    Xg, eg = oracle.safe_gsolve(U, I, s, B, nb)
    Xs, es = oracle.safe_solve(U, s, B, nb)
    assert np.array_equal(Xg, Xs) and np.array_equal(eg, es)


def test_identity_v_safe_with_scaling_bitwise():
    m = 256
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, 9)
    B = W.cn(g, (m, 12))
    shifts = np.diag(T)[g.permutation(m)[:12]] + 1e-9
    I = np.asfortranarray(np.eye(m, dtype=np.complex128))
    Xg, eg = oracle.safe_gsolve(T, I, shifts, B, 32)
    Xs, es = oracle.safe_solve(T, shifts, B, 32)
    assert es.max() > 0
    assert np.array_equal(Xg, Xs) and np.array_equal(eg, es)


def test_scaled_identity_v_is_the_solve_with_scaled_shifts():
    U, s, B = W.plain_problem(60, 6, seed=310)
    c = 0.75
    V = np.asfortranarray(c * np.eye(60, dtype=np.complex128))
    assert np.array_equal(oracle.gsolve(U, V, s, B), oracle.solve(U, s * c, B))


@pytest.mark.parametrize("m", [1, 8, 33, 64])
def test_plain_against_dense_solve(m):
    g, U, V = gen_pair(m, 320 + m)
    s = W.disk(g, 5, 0.5)
    B = np.asfortranarray(W.cn(g, (m, 5)))
    X = oracle.gsolve(U, V, s, B)
    for j in range(5):
        A = np.triu(U) - s[j] * np.triu(V)
        x = np.linalg.solve(A, B[:, j])
        kappa = np.linalg.cond(A, np.inf)
        assert np.abs(X[:, j] - x).max() <= 32 * m * EPS * kappa * np.abs(x).max()


def test_diagonal_closed_form():
    g = W.rng(0, 330)
    m = 20
    U = np.asfortranarray(np.diag(W.disk(g, m, 1.0)))
    V = np.asfortranarray(np.diag(1.0 + 0.5 * W.disk(g, m, 1.0)))
    s = W.disk(g, 4, 0.3)
    B = np.asfortranarray(W.cn(g, (m, 4)))
    X = oracle.gsolve(U, V, s, B)
    ref = B / (np.diag(U)[:, None] - s[None, :] * np.diag(V)[:, None])
    assert np.abs(X - ref).max() <= 4 * EPS * np.abs(ref).max()


def test_safe_invariants_and_plain_agreement():
    g, U, V = gen_pair(150, 340)
    s = W.disk(g, 8, 0.8)
    B = np.asfortranarray(W.cn(g, (150, 8)))
    X, e = oracle.safe_gsolve(U, V, s, B, 32)
    sc = np.ldexp(1.0, -e.astype(np.int64))
    assert np.isfinite(X).all() and (sc <= 1).all()
    Xp = oracle.gsolve(U, V, s, B)
    for j in range(8):
        A = np.triu(U) - s[j] * np.triu(V)
        r = A @ X[:, j] - sc[j] * B[:, j]
        eta = np.abs(r).max() / (np.abs(A).sum(1).max() * np.abs(X[:, j]).max() + sc[j] * np.abs(B[:, j]).max())
        assert eta <= 64 * 150 * EPS
        if e[j] == 0:
            assert np.abs(X[:, j] - Xp[:, j]).max() <= 1e-10 * np.abs(Xp[:, j]).max()


def test_gtrevc_identity_s_is_trevc():
    T = W.trevc_problem(200, seed=7)
    I = np.asfortranarray(np.eye(200, dtype=np.complex128))
    Zg, lam, eg, scg = oracle.gtrevc(T, I, 32)
    Z, e, sc = oracle.trevc(T, 32)
    assert np.array_equal(lam, np.diag(T))
    assert np.array_equal(eg, e) and np.array_equal(Zg, Z)


@pytest.mark.parametrize("m", [60, 180])
def test_gtrevc_residual_and_directions(m):
    g = W.rng(0, 350 + m)
    A = W.cn(g, (m, m))
    Bm = W.cn(g, (m, m)) + 3 * np.eye(m)
    AA, BB, Q, Zq = scipy.linalg.qz(A, Bm, output="complex")
    Z, lam, e, sc = oracle.gtrevc(np.asfortranarray(AA), np.asfortranarray(BB), 32)
    assert np.array_equal(np.diag(Z).real, sc)
    # generalized eigen-residual of the triangular pair
    for j in range(m):
        z = Z[:, j]
        r = AA @ z - lam[j] * (BB @ z)
        assert np.linalg.norm(r) <= 64 * m * EPS * (np.linalg.norm(AA) + abs(lam[j]) * np.linalg.norm(BB)) * np.linalg.norm(z)
    # eigenvectors of the pencil (A, B): X = Zq Z, directions against scipy
    X = Zq @ Z
    X = X / np.linalg.norm(X, axis=0)
    w, Vs = scipy.linalg.eig(A, Bm)
    for j in range(0, m, 9):
        k = int(np.argmin(np.abs(w - lam[j])))
        c = abs(np.vdot(Vs[:, k], X[:, j])) / np.linalg.norm(Vs[:, k])
        assert c >= 1 - 1e-8


def test_gtrevc_columns_entry_point_is_bit_identical():
    g = W.rng(0, 360)
    m = 150
    T = np.asfortranarray(np.triu(W.cn(g, (m, m))) * 3 + np.diag(W.disk(g, m, 1.0)))
    S = np.asfortranarray(np.triu(W.cn(g, (m, m))) * 0.1 + np.diag(1.0 + 0.1 * W.disk(g, m, 1.0)))
    Z, lam, e, _ = oracle.gtrevc(T, S, 32)
    cols = np.array([0, 1, 37, 64, 100, 149])
    Zc, lc, ec = oracle.gtrevc_columns(T, S, cols, 32)
    assert np.array_equal(Zc, Z[:, cols]) and np.array_equal(lc, lam[cols]) and np.array_equal(ec, e[cols])
