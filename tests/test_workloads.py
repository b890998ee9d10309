"""Checks of the synthetic input generators that stand in for the paper's
matrices (no solver arithmetic): the Fox-Li discretisation, the scaling-study
Hermitian matrices and the triangular pencil."""
import numpy as np

from paper_1607_01477_gb300 import workloads as W


def test_fox_li_is_complex_symmetric_and_a_contraction():
    A = W.fox_li(100, 10.0)
    assert np.array_equal(A, A.T)                      # complex symmetric, exactly
    assert not np.allclose(A, A.conj().T)              # and far from Hermitian (nonnormal)
    lam = np.linalg.eigvals(A)
    assert np.abs(lam).max() < 1.0


def test_fox_li_quadrature_converges():
    """The leading eigenvalues are those of the integral operator: they agree
    between n = 100 and n = 200 quadrature points."""
    l1 = np.linalg.eigvals(W.fox_li(100, 10.0))
    l2 = np.linalg.eigvals(W.fox_li(200, 10.0))
    top1 = l1[np.argsort(-np.abs(l1))[:5]]
    top2 = l2[np.argsort(-np.abs(l2))[:5]]
    assert np.abs(top1 - top2).max() <= 1e-9


def test_scaling_problem_spectrum_and_shifts():
    U, s, B = W.scaling_problem(200, 64, seed=3)
    H = np.triu(U) + np.triu(U, 1).conj().T
    lam = np.linalg.eigvalsh(H)
    assert lam.min() >= 1.0 - 1e-12 and lam.max() <= 2.0 + 1e-12
    assert (np.abs(s - 1.5) <= 0.5).all()
    assert (np.tril(U, -1) == 0).all() and B.shape == (200, 64)


def test_pencil_problem_shapes():
    T, S = W.pencil_problem(64, seed=1)
    assert (np.tril(T, -1) == 0).all() and (np.tril(S, -1) == 0).all()
    assert (np.abs(np.diag(S) - 1.0) <= 0.1 + 1e-15).all()
