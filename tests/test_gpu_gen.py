"""GPU parity of the generalized multi-shift solves (appendix, Alg. 8-10)
against the oracle: plain and safe solves, GeneralizedTriangEig, the
generalized Eig driver, and the reduction to the standard GPU solve (V = I,
bitwise)."""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import EPS, to_dev, to_np

pytestmark = pytest.mark.gpu


def gen_pair(m, seed):
    g = W.rng(0, seed)
    U = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(W.disk(g, m, 1.0)))
    V = np.asfortranarray(np.triu(W.cn(g, (m, m))) / np.sqrt(m) + np.diag(1.0 + 0.2 * W.disk(g, m, 1.0)))
    return g, U, V


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,n,nb", [(1, 1, 32), (37, 5, 16), (200, 24, 32), (300, 40, 64), (700, 33, 32)])
def test_plain_matches_oracle(m, n, nb, tensor):
    g, U, V = gen_pair(m, 400 + m)
    s = W.disk(g, n, 0.6)
    B = np.asfortranarray(W.cn(g, (m, n)))
    X = to_dev(B)
    msts.msts_gsolve(to_dev(U), to_dev(V), to_dev(s), X, nb=nb, tensor=tensor)
    Xo = oracle.gsolve(U, V, s, B)
    Xg = to_np(X)
    for j in range(n):
        A = np.triu(U) - s[j] * np.triu(V)
        kappa = np.linalg.cond(A, np.inf) if m <= 300 else 1e6
        err = np.abs(Xg[:, j] - Xo[:, j]).max() / np.abs(Xo[:, j]).max()
        assert err <= max(16 * m * EPS * kappa, 1e-13)


@pytest.mark.parametrize("safe", [False, True])
@pytest.mark.parametrize("m,n,nb", [(96, 10, 16), (256, 64, 32), (300, 17, 64)])
def test_identity_v_reproduces_the_standard_gpu_solve_bitwise(m, n, nb, safe):
    U, s, B = W.plain_problem(m, n, seed=500 + m)
    I = np.asfortranarray(np.eye(m, dtype=np.complex128))
    X1, X2 = to_dev(B), to_dev(B)
    _, sc1, se1, _ = msts.msts_solve(to_dev(U), to_dev(s), X1, safe=safe, nb=nb)
    _, sc2, se2, _ = msts.msts_gsolve(to_dev(U), to_dev(I), to_dev(s), X2, safe=safe, nb=nb)
    assert torch.equal(X1, X2)
    if safe:
        assert torch.equal(se1, se2)


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(256, 32), (300, 16), (320, 64)])
def test_safe_with_scaling_matches_oracle(m, nb, tensor):
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, 11)
    S = np.asfortranarray(np.triu(W.cn(g, (m, m))) * 0.1 + np.diag(1.0 + 0.1 * W.disk(g, m, 1.0)))
    lam = np.diag(T) / np.diag(S)
    B = W.cn(g, (m, 24))
    shifts = lam[g.permutation(m)[:24]] * (1 + 1e-9)
    X = to_dev(B)
    _, sc, se, st = msts.msts_gsolve(to_dev(T), to_dev(S), to_dev(shifts), X, safe=True, nb=nb, tensor=tensor)
    Xo, eo = oracle.safe_gsolve(T, S, shifts, B, nb)
    eg = to_np(se)
    assert eo.max() > 0
    assert np.array_equal(eg, eo)
    Xg = to_np(X)
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(1, 32), (97, 16), (300, 32), (640, 64)])
def test_gtrevc_matches_oracle(m, nb, tensor):
    g = W.rng(0, 600 + m)
    A = W.cn(g, (m, m))
    Bm = W.cn(g, (m, m)) + 3 * np.eye(m)
    T, S, _, _ = scipy.linalg.qz(A, Bm, output="complex")
    T, S = np.asfortranarray(T), np.asfortranarray(S)
    Z, lam, sc, se, st = msts.msts_gtrevc(to_dev(T), to_dev(S), nb=nb, tensor=tensor)
    Zo, lo_, eo, sco = oracle.gtrevc(T, S, nb)
    assert np.array_equal(to_np(lam), lo_)
    assert np.array_equal(to_np(se), eo)
    Zg = to_np(Z)
    assert (np.tril(Zg, -1) == 0).all()
    scale = np.maximum(np.abs(Zo).max(axis=0), 1e-300)
    assert (np.abs(Zg - Zo).max(axis=0) / scale).max() <= 1e-8
    Td, Sd = torch.triu(to_dev(T)), torch.triu(to_dev(S))
    zs = Z / Z.abs().amax(dim=0, keepdim=True)
    R = Td @ zs - (Sd @ zs) * lam[None, :]
    nrm = torch.linalg.norm(Td) + lam.abs()[None, :] * torch.linalg.norm(Sd)
    rho = torch.linalg.norm(R, dim=0) / (nrm[0] * torch.linalg.norm(zs, dim=0))
    assert rho.max().item() <= 4 * m * EPS


@pytest.mark.parametrize("tensor", [False, True])
def test_identity_v_tensor_path_matches_the_standard_tensor_solve(tensor):
    """With V = I the generalized tensor-core update ([U | I] against
    [X; -s X]) computes the standard update to FP64 accuracy (its digit planes
    differ, so not bitwise): forward difference within the kappa bound."""
    m, n, nb = 300, 40, 32
    U, s, B = W.plain_problem(m, n, seed=530)
    I = np.asfortranarray(np.eye(m, dtype=np.complex128))
    X1, X2 = to_dev(B), to_dev(B)
    msts.msts_solve(to_dev(U), to_dev(s), X1, nb=nb, tensor=tensor)
    msts.msts_gsolve(to_dev(U), to_dev(I), to_dev(s), X2, nb=nb, tensor=True)
    X1n, X2n = to_np(X1), to_np(X2)
    for j in range(n):
        A = np.triu(U) - s[j] * np.eye(m)
        kappa = np.linalg.cond(A, np.inf)
        assert np.abs(X1n[:, j] - X2n[:, j]).max() <= 16 * m * EPS * kappa * np.abs(X1n[:, j]).max()


@pytest.mark.parametrize("tensor", [False, True])
def test_gtrevc_full_size_sampled(tensor):
    """GeneralizedTriangEig of the 4096 synthetic pencil (the size bench.py
    times): 12 sampled columns against the oracle's column entry point
    (lambda bitwise, exponents equal, Z within 1e-8) and the generalized
    residual of every 64th column."""
    T, S = W.pencil_problem(4096)
    Td, Sd = to_dev(T), to_dev(S)
    Z, lam, sc, se, st = msts.msts_gtrevc(Td, Sd, nb=32, tensor=tensor)
    cols = np.linspace(1, 4095, 12).astype(int)
    Zo, lo_, eo = oracle.gtrevc_columns(T, S, cols, 32)
    assert np.array_equal(to_np(lam)[cols], lo_)
    assert np.array_equal(to_np(se)[cols], eo)
    Zg = to_np(Z[:, torch.from_numpy(cols).to(Z.device)])
    rel = np.abs(Zg - Zo).max(axis=0) / np.abs(Zo).max(axis=0)
    assert rel.max() <= 1e-8
    sample = torch.arange(0, 4096, 64, device=Td.device)
    zs = Z[:, sample] / Z[:, sample].abs().amax(dim=0, keepdim=True)
    R = torch.triu(Td) @ zs - (torch.triu(Sd) @ zs) * lam[sample][None, :]
    rho = torch.linalg.norm(R, dim=0) / ((torch.linalg.norm(Td) + lam[sample].abs() * torch.linalg.norm(Sd))
                                         * torch.linalg.norm(zs, dim=0))
    assert rho.max().item() <= 4 * 4096 * EPS


@pytest.mark.parametrize("m", [50, 400])
def test_geig_driver_residual(m):
    g = W.rng(0, 700 + m)
    A = W.cn(g, (m, m))
    Bm = W.cn(g, (m, m)) + 3 * np.eye(m)
    lam, X, st = msts.geig(A, Bm, nb=32)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda()
    R = Ad @ X - (Bd @ X) * lam[None, :]
    res = torch.linalg.norm(R) / (torch.linalg.norm(Ad) + lam.abs().max() * torch.linalg.norm(Bd))
    assert res.item() <= 1e-13
    w = scipy.linalg.eigvals(A, Bm)
    assert np.abs(np.sort_complex(w) - np.sort_complex(lam.cpu().numpy())).max() <= 1e-9 * np.abs(w).max()
