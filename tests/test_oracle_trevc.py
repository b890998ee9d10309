"""Pins for the oracle's triangular eigenvectors (Alg. 6, Sec. 4)."""
import numpy as np
import pytest

import oracle
from paper_1607_01477_gb300 import workloads as W
from conftest import EPS


def eig_residuals(T, Z):
    """rho_j = ||T z_j - lambda_j z_j||_2 / (||T||_F ||z_j||_2), z_j rescaled to max|z| = 1."""
    Tu = np.triu(T)
    lam = np.diag(Tu)
    fro = np.linalg.norm(Tu)
    zs = Z / np.abs(Z).max(axis=0, keepdims=True)
    R = Tu @ zs - zs * lam[None, :]
    return np.linalg.norm(R, axis=0) / (fro * np.linalg.norm(zs, axis=0))


def test_two_by_two_closed_form():
    """T = [[a, b], [0, c]]: z_1 = e_1 and z_2 = [b/(c-a), 1] (Eq. triangeig-2 with s = 1)."""
    a, b, c = 0.3 + 0.2j, -1.7 + 0.4j, -0.5 + 0.9j
    T = np.asfortranarray(np.array([[a, b], [0, c]], dtype=np.complex128))
    Z, e, sc = oracle.trevc(T, 32)
    assert (e == 0).all() and (sc == 1).all()
    assert Z[0, 0] == 1 and Z[1, 0] == 0 and Z[1, 1] == 1
    assert abs(Z[0, 1] - b / (c - a)) <= 4 * EPS * abs(b / (c - a))


@pytest.mark.parametrize("m,nb", [(3, 32), (12, 4), (40, 8), (70, 32)])
def test_directions_match_numpy_eig(m, nb):
    """Well-separated eigenvalues: each z_j is parallel to numpy.linalg.eig's vector."""
    g = W.rng(0, 77 + m)
    d = np.exp(2j * np.pi * np.arange(m) / m) * (1 + 0.3 * g.random(m))
    T = W.upper(g, m, d, 0.3)
    Z, e, sc = oracle.trevc(T, nb)
    w, V = np.linalg.eig(np.triu(T))
    for j in range(m):
        k = np.argmin(np.abs(w - T[j, j]))
        v = V[:, k]
        z = Z[:, j]
        c = np.vdot(v, z) / np.vdot(v, v)
        assert np.linalg.norm(z - c * v) <= 1e-9 * np.linalg.norm(z)


@pytest.mark.parametrize("m,nb", [(200, 32), (257, 16), (600, 32)])
def test_structure_scales_and_residual(m, nb):
    """Z upper triangular with diag(Z) = s = 2^-e, and a small eigen-residual even
    with clustered eigenvalues (spacing 1e-10) and scaling exercised."""
    T = W.trevc_problem(m, seed=m)
    Z, e, sc = oracle.trevc(T, nb)
    assert (np.tril(Z, -1) == 0).all()
    assert np.array_equal(np.diag(Z).real, np.ldexp(1.0, -e.astype(np.int64)))
    assert np.array_equal(sc, np.ldexp(1.0, -e.astype(np.int64)))
    assert np.isfinite(Z).all()
    rho = eig_residuals(T, Z)
    assert rho.max() <= 2 * m * EPS
    if m >= 600:
        assert e.max() > 0          # overflow scaling was exercised


def test_first_column_is_unit():
    T = W.trevc_problem(33, seed=2)
    Z, e, sc = oracle.trevc(T, 8)
    assert Z[0, 0] == 1 and (Z[1:, 0] == 0).all()


def test_selected_columns_match_full_trevc():
    """The per-column entry point repeats or_trevc's arithmetic bit for bit."""
    T = W.trevc_problem(300, seed=9)
    Z, e, sc = oracle.trevc(T, 32)
    cols = [0, 1, 31, 32, 33, 150, 299]
    Zc, ec = oracle.trevc_columns(T, cols, 32)
    assert np.array_equal(ec, e[cols])
    assert np.array_equal(Zc, Z[:, cols])


def test_full_size_workload_sampled_columns():
    """The 4096 x 4096 TREVC workload (the benchmark's matrix): 48 sampled
    columns, among them members of eigenvalue clusters (spacing 1e-10) and the
    last columns, whose growth drives e_j into the thousands (scales far below
    the double range).  Each column is zero below its diagonal entry 2^-e_j and
    has eigen-residual <= 2 m eps."""
    T = W.trevc_problem(4096)
    m = T.shape[0]
    lam = np.diag(T)
    gap = np.array([np.partition(np.abs(lam - lam[j]), 1)[1] for j in range(m)])
    clustered = np.flatnonzero(gap < 1e-9)
    assert clustered.size >= 150
    g = W.rng(0, 4096)
    cols = np.unique(np.concatenate([[0, 1, 31, 32, 33], clustered[:8], clustered[-8:],
                                     g.choice(m, 24, replace=False), [m - 3, m - 2, m - 1]]))
    Zc, ec = oracle.trevc_columns(T, cols, 32)
    Tu = np.triu(T)
    fro = np.linalg.norm(Tu)
    for k, j in enumerate(cols):
        z = Zc[:, k]
        assert z[j] == np.ldexp(1.0, -int(ec[k]))
        assert (z[j + 1:] == 0).all() and np.isfinite(z).all()
        zs = z / np.abs(z).max()
        rho = np.linalg.norm(Tu @ zs - lam[j] * zs) / (fro * np.linalg.norm(zs))
        assert rho <= 2 * m * EPS, (j, rho)
    assert ec.max() >= 1000
