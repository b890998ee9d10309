"""Pins of the oracle's 1-norm pseudospectra (footnote to Sec. 5: Hager's
estimator with Higham's refinements, shifted triangular solves at the grid
points) and of the automatic spectral-portrait grid, against dense inverses,
closed forms and the estimator's own guarantees."""
import numpy as np
import pytest

import oracle
from paper_1607_01477_gb300 import workloads as W

EPS = np.finfo(np.float64).eps


def tri_problem(m, seed, N=40):
    g = W.rng(0, seed)
    T = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(W.disk(g, m, 1.0)))
    z = W.disk(g, N, 1.5)
    return g, T, z


def dense_resolvent(T, z, Q=None):
    m = T.shape[0]
    R = np.linalg.inv(np.triu(T) - z * np.eye(m))
    return R if Q is None else Q @ R @ Q.conj().T


def alt_vector(m):
    i = np.arange(m)
    return np.where(i % 2 == 0, 1.0, -1.0) * (1.0 + i / (m - 1))


@pytest.mark.parametrize("use_q", [False, True])
@pytest.mark.parametrize("m", [2, 17, 60])
def test_estimate_is_attained_by_the_reported_vector(m, use_q):
    """The estimate is the 1-norm of R applied to the vector the estimator
    reports (a column e_j, the start vector e/m, or 2/(3m) times the
    alternative vector) -- computed here from the dense resolvent, so a
    misplaced Q or Q^H, a wrong shift sign or a dropped term fails."""
    g, T, z = tri_problem(m, 40 + m)
    Q = np.asfortranarray(np.linalg.qr(W.cn(g, (m, m)))[0]) if use_q else None
    est, kind, steps = oracle.pseudospectra_1norm(T, z, Q)
    assert (steps >= 1).all() and (steps <= 5).all()
    for p in range(z.size):
        R = dense_resolvent(T, z[p], Q)
        if kind[p] >= 0:
            ref = np.abs(R[:, kind[p]]).sum()
        elif kind[p] == -1:
            ref = np.abs(R @ (np.ones(m) / m)).sum()
        else:
            assert kind[p] == -2
            ref = 2.0 * np.abs(R @ alt_vector(m)).sum() / (3 * m)
        assert abs(est[p] - ref) <= 1e-11 * ref


@pytest.mark.parametrize("use_q", [False, True])
def test_lower_bound_and_quality(use_q):
    m = 80
    g, T, z = tri_problem(m, 41, N=60)
    Q = np.asfortranarray(np.linalg.qr(W.cn(g, (m, m)))[0]) if use_q else None
    est, kind, steps = oracle.pseudospectra_1norm(T, z, Q)
    exact = np.array([np.abs(dense_resolvent(T, zz, Q)).sum(axis=0).max() for zz in z])
    assert (est <= exact * (1 + 1e-10)).all()          # an estimate of ||R||_1 from below
    assert (est >= 0.3 * exact).all()                  # Hager/Higham: within a small factor in practice
    assert np.median(est / exact) >= 0.9


def test_diagonal_matrix_is_exact():
    """R diagonal: the gradient step picks the largest |1/(d_i - z)|, which is
    the 1-norm, so the estimate is exact."""
    g = W.rng(0, 42)
    m = 25
    d = W.disk(g, m, 1.0)
    T = np.asfortranarray(np.diag(d))
    z = W.disk(g, 30, 1.5)
    est, kind, _ = oracle.pseudospectra_1norm(T, z)
    exact = (1.0 / np.abs(d[:, None] - z[None, :])).max(axis=0)
    assert np.abs(est - exact).max() <= 4 * EPS * exact.max()
    assert (kind == np.abs(d[:, None] - z[None, :]).argmin(axis=0)).all()


def test_one_by_one():
    T = np.asfortranarray(np.array([[0.3 + 0.4j]]))
    z = np.array([1.0 + 0.0j, -2.0 + 1.0j])
    est, kind, steps = oracle.pseudospectra_1norm(T, z)
    assert np.abs(est - 1.0 / np.abs(T[0, 0] - z)).max() <= 2 * EPS
    assert (steps == 0).all() and (kind == -1).all()


def test_permutation_similarity_keeps_the_estimate():
    """Q = P (a permutation): Q R Q^H is R with rows and columns permuted alike,
    so its 1-norm and every gradient step of the estimator carry over (the
    start vector e/m and the unit vectors map to themselves): same steps, the
    column index mapped, and the same estimate wherever the alternative vector
    (not permutation-invariant) did not win."""
    m = 50
    g, T, z = tri_problem(m, 43)
    perm = g.permutation(m)
    P = np.zeros((m, m))
    P[perm, np.arange(m)] = 1.0                       # P e_k = e_perm[k]
    Q = np.asfortranarray(P.astype(np.complex128))
    e0, k0, s0 = oracle.pseudospectra_1norm(T, z)
    e1, k1, s1 = oracle.pseudospectra_1norm(T, z, Q)
    assert (s1 == s0).all()
    grad = (k0 != -2) & (k1 != -2)
    assert grad.sum() >= 0.75 * z.size
    assert np.abs(e1 - e0)[grad].max() <= 1e-13 * e0.max()
    col = grad & (k0 >= 0)
    assert (k1[col] == perm[k0[col]]).all() and (k1[grad & (k0 == -1)] == -1).all()


def test_portrait_grid_properties():
    g = W.rng(0, 44)
    m = 30
    d = 0.5 + 2.0 * W.disk(g, m, 1.0)
    T = np.asfortranarray(np.diag(d) + np.triu(W.cn(g, (m, m)), 1))
    nx, ny = 9, 7
    z, box = oracle.portrait_grid(T, nx, ny)
    a, b, c, dd = d.real.min(), d.real.max(), d.imag.min(), d.imag.max()
    h = 0.25 * max(b - a, dd - c)
    assert np.allclose(box, [a - h, b + h, c - h, dd + h], rtol=0, atol=4 * EPS * 4)
    Z = z.reshape(ny, nx)                              # row l: fixed imaginary part
    assert np.array_equal(Z[:, 0].real, np.full(ny, box[0])) and np.array_equal(Z[0, :].imag, np.full(nx, box[2]))
    assert np.abs(Z[:, -1].real - box[1]).max() <= 8 * EPS * abs(box[1]) + 8 * EPS
    assert np.abs(Z[-1, :].imag - box[3]).max() <= 8 * EPS * abs(box[3]) + 8 * EPS
    assert np.ptp(np.diff(Z.real, axis=1)) <= 16 * EPS * np.abs(box).max()
    assert (d.real > box[0]).all() and (d.real < box[1]).all()
    assert (d.imag > box[2]).all() and (d.imag < box[3]).all()


def test_portrait_grid_degenerate_spectrum():
    T = np.asfortranarray(np.eye(4, dtype=np.complex128) * (3.0 - 4.0j))
    z, box = oracle.portrait_grid(T, 3, 3)
    h = 4.0 * 2.0 ** -20                               # 2^-20 max(|Re|, |Im|)
    assert np.array_equal(box, [3.0 - h, 3.0 + h, -4.0 - h, -4.0 + h])
    assert z[4] == 3.0 - 4.0j                          # the centre point of a 3 x 3 grid


def test_alternative_vector_estimate_when_it_wins():
    """Higham's alternative vector x(i) = (-1)^i (1 + i/(m-1)), i = 0..m-1: on
    small problems where it beats Hager's steps (kind -2), the estimate is
    exactly 2 ||R x||_1 / (3m) with R = (T - zI)^{-1} from a dense inverse, and
    it stays a lower bound of ||R||_1.  The inputs are seeded random triangles
    on which the branch is taken (it rarely is)."""
    wins = 0
    for seed in (189, 228, 267, 369, 390):
        g = W.rng(0, 5000 + seed)
        m = int(g.integers(2, 9))
        d = W.disk(g, m, 1.0)
        T = W.upper(g, m, d, [0.3, 3.0, 30.0][seed % 3])
        z = W.disk(g, 6, 1.2)
        est, kind, steps = oracle.pseudospectra_1norm(T, z)[:3]
        x = np.array([(-1.0) ** i * (1.0 + i / (m - 1)) for i in range(m)])
        for p in range(z.size):
            R = np.linalg.inv(np.triu(T) - z[p] * np.eye(m))
            assert est[p] <= np.abs(R).sum(axis=0).max() * (1 + 1e-12)
            if kind[p] == -2:
                wins += 1
                assert est[p] == pytest.approx(2.0 * np.abs(R @ x).sum() / (3.0 * m), rel=1e-10, abs=0)
    assert wins >= 3
