"""Pins of the oracle's other triangular variants (footnote to Sec. 2: the
lower-triangular and right-hand cases): M_j = op(A) - s_j I with op in
{N, T, C} and A upper or lower, solved from the left (columns of B) or the
right (rows of B); plain and safe (Alg. 5 in the variant's substitution
order).  Pinned against dense solves, closed forms, the upper solve through
exact reversal and transposition identities, and safe invariants."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1607_01477_gb300 import workloads as W

EPS = np.finfo(np.float64).eps
OMEGA = 2.0 ** 960
VARIANTS = list(itertools.product(["left", "right"], ["upper", "lower"], ["N", "T", "C"]))


def tri(A, uplo):
    return np.triu(A) if uplo == "upper" else np.tril(A)


def op(A, trans):
    return A if trans == "N" else (A.T if trans == "T" else A.conj().T)


def random_tri(g, m, uplo):
    """Well-conditioned random triangle: off-diagonal CN/sqrt(m), unit-disk
    diagonal pushed away from the shifts."""
    A = W.cn(g, (m, m)) / np.sqrt(m)
    A[np.arange(m), np.arange(m)] = 3.0 + W.disk(g, m, 1.0)
    return np.asfortranarray(tri(A, uplo))


def rhs(g, m, n, side):
    return np.asfortranarray(W.cn(g, (m, n) if side == "left" else (n, m)))


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_against_dense_solve(side, uplo, trans):
    g = W.rng(0, 800)
    m, n = 45, 6
    A = random_tri(g, m, uplo)
    s = W.disk(g, n, 1.0)
    B = rhs(g, m, n, side)
    X = oracle.solve_variant(A, s, B, side, uplo, trans)
    for j in range(n):
        M = op(tri(A, uplo), trans) - s[j] * np.eye(m)
        if side == "left":
            x, got = np.linalg.solve(M, B[:, j]), X[:, j]
        else:
            x, got = np.linalg.solve(M.T, B[j, :]), X[j, :]
        kappa = np.linalg.cond(M, np.inf)
        assert np.abs(got - x).max() <= 32 * m * EPS * kappa * np.abs(x).max()


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_only_the_named_triangle_is_read(side, uplo, trans):
    g = W.rng(0, 801)
    m, n = 30, 4
    A = random_tri(g, m, uplo)
    junk = W.cn(g, (m, m)) * 1e3
    Aj = np.asfortranarray(A + (np.tril(junk, -1) if uplo == "upper" else np.triu(junk, 1)))
    s = W.disk(g, n, 1.0)
    B = rhs(g, m, n, side)
    assert np.array_equal(oracle.solve_variant(A, s, B, side, uplo, trans),
                          oracle.solve_variant(Aj, s, B, side, uplo, trans))


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_diagonal_closed_form(side, uplo, trans):
    g = W.rng(0, 802)
    m, n = 12, 5
    d = 2.0 + W.disk(g, m, 1.0)
    A = np.asfortranarray(np.diag(d))
    s = W.disk(g, n, 0.5)
    B = rhs(g, m, n, side)
    X = oracle.solve_variant(A, s, B, side, uplo, trans)
    dd = d.conj() if trans == "C" else d
    piv = dd[:, None] - s[None, :]
    ref = B / piv if side == "left" else B / piv.T
    assert np.abs(X - ref).max() <= 4 * EPS * np.abs(ref).max()


def test_left_upper_n_and_c_are_the_standard_solves_bitwise():
    U, s, B = W.plain_problem(70, 9, seed=803)
    assert np.array_equal(oracle.solve_variant(U, s, B, "left", "upper", "N"), oracle.solve(U, s, B))
    # (U^H - s I) x = b is the conjugate-transposed solve with shifts conj(s)
    assert np.array_equal(oracle.solve_variant(U, s, B, "left", "upper", "C"),
                          oracle.solve(U, s.conj(), B, conj_trans=True))


@pytest.mark.parametrize("trans", ["N", "T", "C"])
def test_lower_is_the_reversed_upper_solve_bitwise(trans):
    """Forward substitution on a lower-triangular operator M is back
    substitution on J M J (J the reversal) with the right-hand side reversed:
    the same products in the same order, hence bitwise equal."""
    g = W.rng(0, 804)
    m, n = 37, 5
    L = random_tri(g, m, "lower")
    s = W.disk(g, n, 1.0)
    B = rhs(g, m, n, "left")
    M = op(L, trans)                                   # upper for T/C, lower for N
    if trans == "N":
        U = np.asfortranarray(M[::-1, ::-1])
        Xr = oracle.solve(U, s, np.asfortranarray(B[::-1, :]))[::-1, :]
    else:
        Xr = oracle.solve(np.asfortranarray(M), s, B)
    assert np.array_equal(oracle.solve_variant(L, s, B, "left", "lower", trans), Xr)


def bidiag_pow2_operator(m, p, d_exp, upper):
    """Effective left operator E (E x = b) with E(i,i) = 2^d and one
    off-diagonal -2^p next to it, b the unit vector where substitution starts:
    x(k) = 2^(-d + (p - d) k) at substitution step k."""
    E = np.zeros((m, m))
    E[np.arange(m), np.arange(m)] = 2.0 ** d_exp
    if upper:
        E[np.arange(m - 1), np.arange(1, m)] = -(2.0 ** p)
        start, steps = m - 1, m - 1 - np.arange(m)
    else:
        E[np.arange(1, m), np.arange(m - 1)] = -(2.0 ** p)
        start, steps = 0, np.arange(m)
    return E, start, -d_exp + (p - d_exp) * steps


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
@pytest.mark.parametrize("nb", [8, 5])
def test_safe_pow2_closed_form_bitwise(side, uplo, trans, nb):
    """Every variant's safe solve on an exact power-of-two bidiagonal operator
    whose solution overflows without scaling: x * 2^e is a power of two known in
    closed form, so the check is bitwise, and the scaled solution stays < Omega."""
    m, p = 32, 1
    M_upper = (uplo == "upper") == (trans == "N")       # triangle of op(A)
    E_upper = M_upper if side == "left" else not M_upper
    E, start, log2x = bidiag_pow2_operator(m, p, -40, E_upper)
    M = E if side == "left" else E.T                    # left: M x = b; right: M^T x = b
    A = np.asfortranarray((M if trans == "N" else M.T).astype(np.complex128))   # real: A^H = A^T
    b = np.zeros(m, dtype=np.complex128)
    b[start] = 1.0
    B = np.asfortranarray(b[:, None] if side == "left" else b[None, :])
    X, e = oracle.safe_solve_variant(A, np.zeros(1, dtype=np.complex128), B, nb, side, uplo, trans)
    x = X[:, 0] if side == "left" else X[0, :]
    assert e[0] > 0 and e[0] >= log2x.max() - 960
    expect = np.array([np.ldexp(1.0, int(k) - int(e[0])) for k in log2x])
    assert np.array_equal(x.real, expect) and (x.imag == 0).all()
    assert np.abs(x).max() < OMEGA


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_safe_invariants_and_plain_agreement(side, uplo, trans):
    g = W.rng(0, 805)
    m, n, nb = 90, 7, 16
    A = random_tri(g, m, uplo)
    s = W.disk(g, n, 1.0)
    B = rhs(g, m, n, side)
    X, e = oracle.safe_solve_variant(A, s, B, nb, side, uplo, trans)
    assert (e == 0).all()
    Xp = oracle.solve_variant(A, s, B, side, uplo, trans)
    assert np.abs(X - Xp).max() <= 1e-12 * np.abs(Xp).max()


def test_safe_scaled_residual_on_clustered_lower_problem():
    """A lower problem that rescales: M x = 2^-e b with a small normwise
    backward error, and x 2^e equal to the plain solution where that is finite."""
    m, n, nb = 200, 10, 32
    T = W.trevc_problem(m, seed=91, cluster_frac=0.1, offdiag_scale=30.0)
    L = np.asfortranarray(T.conj().T)                   # lower, badly scaled off-diagonal
    g = W.rng(0, 806)
    s = np.diag(L)[g.permutation(m)[:n]] + 1e-9
    B = rhs(g, m, n, "left")
    X, e = oracle.safe_solve_variant(L, s, B, nb, "left", "lower", "N")
    assert e.max() > 0 and np.isfinite(X).all()
    sc = np.ldexp(1.0, -e.astype(np.int64))
    for j in range(n):
        M = np.tril(L) - s[j] * np.eye(m)
        r = M @ X[:, j] - sc[j] * B[:, j]
        eta = np.abs(r).max() / (np.abs(M).sum(1).max() * np.abs(X[:, j]).max() + sc[j] * np.abs(B[:, j]).max())
        assert eta <= 64 * m * EPS
    Xp = oracle.solve_variant(L, s, B, "left", "lower", "N")
    for j in range(n):
        if np.isfinite(Xp[:, j]).all():
            up = np.ldexp(X[:, j].real, int(e[j])) + 1j * np.ldexp(X[:, j].imag, int(e[j]))
            assert np.abs(up - Xp[:, j]).max() <= 1e-10 * np.abs(Xp[:, j]).max()
