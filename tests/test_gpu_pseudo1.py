"""GPU parity of the pseudospectra extras against the oracle: 1-norm
pseudospectra (Hager/Higham estimator on multi-shift solves, with and
without Schur vectors Q, both product paths), the automatic portrait grid
(bitwise), and the SpectralPortrait driver on the Fox-Li matrix."""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import EPS, to_dev, to_np

pytestmark = pytest.mark.gpu


def tri_problem(m, N, seed):
    g = W.rng(0, seed)
    T = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(W.disk(g, m, 1.0)))
    z = W.disk(g, N, 1.5)
    return g, T, z


def check_against_oracle(est, kind, steps, eo, ko, so, min_agree=1.0):
    est, kind, steps = to_np(est), to_np(kind), to_np(steps)
    same = (kind == ko) & (steps == so)
    # where both took the same decisions the estimates are the same 1-norm of
    # the same vector, computed in different orders
    assert same.mean() >= min_agree, same.mean()
    assert (np.abs(est - eo)[same] <= 1e-10 * eo[same]).all()
    # elsewhere (a near-tie decided differently) both are valid lower bounds of
    # comparable size
    if (~same).any():
        assert (np.abs(est - eo)[~same] <= 0.5 * eo[~same]).all()


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,N,nb", [(1, 3, 32), (2, 5, 16), (17, 40, 16), (100, 300, 32), (333, 120, 64)])
def test_triangular_matches_oracle(m, N, nb, tensor):
    g, T, z = tri_problem(m, N, 1100 + m)
    est, kind, steps, st = msts.msts_pseudospectra_1norm(to_dev(T), to_dev(z), nb=nb, tensor=tensor)
    eo, ko, so = oracle.pseudospectra_1norm(T, z)
    check_against_oracle(est, kind, steps, eo, ko, so)
    assert int(st.item()) == 0


@pytest.mark.parametrize("tensor", [False, True])
def test_with_schur_vectors_matches_oracle_and_bounds(tensor):
    m, N = 120, 150
    g, T, z = tri_problem(m, N, 1200)
    Q = np.asfortranarray(np.linalg.qr(W.cn(g, (m, m)))[0])
    est, kind, steps, _ = msts.msts_pseudospectra_1norm(to_dev(T), to_dev(z), to_dev(Q), nb=32, tensor=tensor)
    eo, ko, so = oracle.pseudospectra_1norm(T, z, Q)
    check_against_oracle(est, kind, steps, eo, ko, so)
    A = Q @ np.triu(T) @ Q.conj().T
    e = to_np(est)
    for p in range(0, N, 15):
        exact = np.abs(np.linalg.inv(z[p] * np.eye(m) - A)).sum(axis=0).max()
        assert e[p] <= exact * (1 + 1e-10)


def test_diagonal_is_exact():
    g = W.rng(0, 1300)
    m = 64
    d = W.disk(g, m, 1.0)
    z = W.disk(g, 200, 1.5)
    est, kind, _, _ = msts.msts_pseudospectra_1norm(to_dev(np.diag(d)), to_dev(z), tensor=True)
    exact = (1.0 / np.abs(d[:, None] - z[None, :])).max(axis=0)
    assert np.abs(to_np(est) - exact).max() <= 4 * EPS * exact.max()


def test_full_size_pseudospectra_workload_sampled():
    """The pseudospectra workload (2000 x 2000 triangular, 100 x 100 grid on
    [-1.5, 1.5]^2) in the 1-norm on the tensor-core path: 24 sampled points
    against the oracle, and 3 against the dense resolvent."""
    T, z, _ = W.pseudo_problem()
    est, kind, steps, st = msts.msts_pseudospectra_1norm(to_dev(T), to_dev(z), nb=32, tensor=True)
    sample = np.linspace(0, z.size - 1, 24).astype(int)
    eo, ko, so = oracle.pseudospectra_1norm(T, z[sample])
    e, k, s = to_np(est), to_np(kind), to_np(steps)
    check_against_oracle(torch.from_numpy(e[sample]), torch.from_numpy(k[sample]), torch.from_numpy(s[sample]),
                         eo, ko, so, min_agree=0.9)
    for p in sample[::8]:
        exact = np.abs(scipy.linalg.solve_triangular(np.triu(T) - z[p] * np.eye(2000), np.eye(2000))).sum(0).max()
        assert e[p] <= exact * (1 + 1e-10) and e[p] >= 0.3 * exact
    assert (s >= 1).all() and (s <= 5).all()


@pytest.mark.parametrize("nx,ny", [(1, 1), (9, 7), (100, 100), (3, 1)])
def test_portrait_grid_bitwise(nx, ny):
    g = W.rng(0, 1400)
    m = 50
    T = np.asfortranarray(np.triu(W.cn(g, (m, m)), 1) + np.diag(0.3 + 1.7 * W.disk(g, m, 1.0)))
    z, box = msts.msts_portrait_grid(to_dev(T), nx, ny)
    zo, bo = oracle.portrait_grid(T, nx, ny)
    assert np.array_equal(to_np(box), bo)
    assert np.array_equal(to_np(z), zo)


def test_portrait_grid_degenerate_and_single_entry():
    for T in (np.eye(5, dtype=np.complex128) * (3.0 - 4.0j), np.array([[0.0j]])):
        T = np.asfortranarray(T)
        z, box = msts.msts_portrait_grid(to_dev(T), 4, 3)
        zo, bo = oracle.portrait_grid(T, 4, 3)
        assert np.array_equal(to_np(box), bo) and np.array_equal(to_np(z), zo)


def test_spectral_portrait_driver_on_fox_li():
    """SpectralPortrait of the Fox-Li matrix (F = 10, n = 64; Schur factor
    from the host library) on a 50 x 50 automatic grid: the 2-norm portrait
    (64 Lanczos steps: the whole Krylov space) equals 1/sigma_min from the
    dense SVD, and the 1-norm portrait is a lower bound of the dense 1-norm
    within the estimator's usual factor."""
    n = 64
    A = W.fox_li(n, 10.0)
    T, Q = scipy.linalg.schur(A, output="complex")
    Td, Qd = to_dev(np.asfortranarray(T)), to_dev(np.asfortranarray(Q))
    r2, box, _ = msts.spectral_portrait(Td, 50, 50, norm=2, iters=n)
    z, _ = msts.msts_portrait_grid(Td, 50, 50)
    zz = to_np(z).reshape(50, 50)
    R2 = to_np(r2)
    for (l, k) in [(0, 0), (10, 37), (25, 25), (49, 3)]:
        smin = np.linalg.svd(zz[l, k] * np.eye(n) - A, compute_uv=False).min()
        assert abs(R2[l, k] * smin - 1.0) <= 1e-9
    r1, _, _ = msts.spectral_portrait(Td, 50, 50, norm=1, Q=Qd)
    R1 = to_np(r1)
    for (l, k) in [(0, 0), (10, 37), (25, 25), (49, 3)]:
        exact = np.abs(np.linalg.inv(zz[l, k] * np.eye(n) - A)).sum(axis=0).max()
        assert R1[l, k] <= exact * (1 + 1e-9) and R1[l, k] >= 0.3 * exact
