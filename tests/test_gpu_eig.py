"""GPU parity: the back-transformation X = Q Z (Alg. 6 "Eig", Sec. 4) against
the oracle on both product paths, column normalisation, and the Eig driver's
eigen-residual (Schur on the host, TREVC and back-transformation on the GPU),
up to the full 4096 TREVC size."""
import numpy as np
import pytest
import scipy.linalg
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import EPS, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m", [1, 5, 37, 128, 300, 1000])
def test_back_transform_matches_oracle(m, tensor):
    g = W.rng(0, 80 + m)
    Q = np.asfortranarray(W.cn(g, (m, m)))
    Z = np.asfortranarray(W.cn(g, (m, m)) * np.exp(8 * g.standard_normal((1, m))))   # column scales vary
    Xo = oracle.back_transform(Q, Z)
    X, st = msts.msts_back_transform(to_dev(Q), to_dev(Z), tensor=tensor)
    Xg = to_np(X)
    # elementwise bound of two FP64-accurate products: c m eps (|Q| |triu Z|)
    bound = 8 * m * EPS * (np.abs(Q) @ np.abs(np.triu(Z)))
    assert (np.abs(Xg - Xo) <= bound + 1e-300).all()
    assert int(st.item()) == 0


@pytest.mark.parametrize("tensor", [False, True])
def test_normalised_columns(tensor):
    g = W.rng(0, 90)
    m = 200
    Q = np.asfortranarray(W.cn(g, (m, m)))
    Z = np.asfortranarray(np.triu(W.cn(g, (m, m))) * 1e150)
    Z[:, 7] = 0.0                                  # a zero column stays zero
    X, _ = msts.msts_back_transform(to_dev(Q), to_dev(Z), tensor=tensor, normalize=True)
    Xg = to_np(X)
    nrm = np.linalg.norm(Xg, axis=0)
    assert np.all(np.abs(np.delete(nrm, 7) - 1.0) <= 64 * EPS)
    assert np.all(Xg[:, 7] == 0)
    Xo = oracle.back_transform(Q, Z)
    Xo = Xo / np.where(np.linalg.norm(Xo, axis=0) == 0, 1, np.linalg.norm(Xo, axis=0))
    assert np.abs(Xg - Xo).max() <= 1e-12


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m", [64, 300, 700])
def test_eig_driver_residual(m, tensor):
    g = W.rng(0, 100 + m)
    A = W.cn(g, (m, m))
    w, X, st = msts.eig(A, nb=32, tensor=tensor)
    Ad = torch.from_numpy(A).cuda()
    R = Ad @ X - X * w[None, :]
    res = (torch.linalg.norm(R) / torch.linalg.norm(Ad)).item()
    assert res <= 1e-13
    nrm = torch.linalg.norm(X, dim=0).cpu().numpy()
    assert np.all(np.abs(nrm - 1.0) <= 64 * EPS)
    wn = np.linalg.eigvals(A)
    assert np.abs(np.sort_complex(wn) - np.sort_complex(w.cpu().numpy())).max() <= 1e-10 * np.abs(wn).max()


@pytest.mark.parametrize("tensor", [False, True])
def test_full_size_back_transform_of_trevc(tensor):
    """Workload 2 (4096, clustered eigenvalues): Z from msts_trevc, a random
    unitary Q, X = Q Z normalised; A = Q T Q^H must satisfy A X = X diag(T)."""
    T = W.trevc_problem()
    Td = to_dev(T)
    Z, sc, se, st = msts.msts_trevc(Td, nb=32, tensor=tensor)
    g = torch.Generator(device="cuda").manual_seed(1607)
    G = torch.randn((4096, 4096), dtype=torch.complex128, device="cuda", generator=g)
    Qd, _ = torch.linalg.qr(G)
    Qd = msts.colmajor(Qd)
    X, st2 = msts.msts_back_transform(Qd, Z, tensor=tensor, normalize=True)
    Tu = torch.triu(Td)
    A = Qd @ Tu @ Qd.conj().T
    lam = torch.diagonal(Tu)
    res = (torch.linalg.norm(A @ X - X * lam[None, :]) / torch.linalg.norm(A)).item()
    assert res <= 1e-13
