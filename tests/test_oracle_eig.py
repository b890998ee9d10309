"""Pins of the oracle's back-transformation X = Q triu(Z) (Alg. 6 "Eig", Sec. 4):
closed forms for identity, permutation and diagonal Q, invariance under a
unitary Q, and the eigen-residual of the full Eig path (Schur from scipy, the
oracle's TREVC, then the back-transformation)."""
import numpy as np
import scipy.linalg

import oracle
from paper_1607_01477_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def rand_z(g, m):
    return np.asfortranarray(W.cn(g, (m, m)))


def test_identity_q_returns_upper_triangle_exactly():
    g = W.rng(0, 70)
    Z = rand_z(g, 23)
    X = oracle.back_transform(np.asfortranarray(np.eye(23, dtype=np.complex128)), Z)
    assert np.array_equal(X, np.triu(Z))


def test_permutation_q_permutes_rows_exactly():
    g = W.rng(0, 71)
    m = 31
    Z = rand_z(g, m)
    p = g.permutation(m)
    Q = np.zeros((m, m), dtype=np.complex128, order="F")
    Q[np.arange(m), p] = 1.0                     # row i of X = row p[i] of triu(Z)
    X = oracle.back_transform(Q, Z)
    assert np.array_equal(X, np.triu(Z)[p, :])


def test_only_the_upper_triangle_of_z_is_read():
    g = W.rng(0, 72)
    m = 17
    Q = rand_z(g, m)
    Z = rand_z(g, m)
    Zt = np.asfortranarray(np.triu(Z))
    assert np.array_equal(oracle.back_transform(Q, Z), oracle.back_transform(Q, Zt))


def test_diagonal_q_scales_rows():
    g = W.rng(0, 73)
    m = 40
    ph = np.exp(2j * np.pi * g.random(m))
    Q = np.asfortranarray(np.diag(ph))
    Z = rand_z(g, m)
    X = oracle.back_transform(Q, Z)
    ref = ph[:, None] * np.triu(Z)
    assert np.abs(X - ref).max() <= 2 * EPS * np.abs(Z).max()


def test_unitary_q_preserves_frobenius_norm():
    g = W.rng(0, 74)
    m = 90
    Q, _ = np.linalg.qr(W.cn(g, (m, m)))
    Q = np.asfortranarray(Q)
    Z = rand_z(g, m)
    X = oracle.back_transform(Q, Z)
    assert abs(np.linalg.norm(X) / np.linalg.norm(np.triu(Z)) - 1.0) <= 64 * m * EPS


def test_eig_path_residual_and_directions():
    g = W.rng(0, 75)
    m = 120
    A = W.cn(g, (m, m))
    T, Q = scipy.linalg.schur(A, output="complex")
    Z, e, sc = oracle.trevc(np.asfortranarray(T), 32)
    X = oracle.back_transform(np.asfortranarray(Q), Z)
    X = X / np.linalg.norm(X, axis=0)
    w = np.diag(T)
    res = np.linalg.norm(A @ X - X * w[None, :]) / np.linalg.norm(A)
    assert res <= 1e-13
    wn, Vn = np.linalg.eig(A)
    for j in range(0, m, 7):
        k = int(np.argmin(np.abs(wn - w[j])))
        c = abs(np.vdot(Vn[:, k], X[:, j])) / (np.linalg.norm(Vn[:, k]) * np.linalg.norm(X[:, j]))
        assert c >= 1 - 1e-9
