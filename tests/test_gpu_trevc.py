"""GPU parity: safe triangular eigenvectors (Alg. 6) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import EPS, to_dev, to_np

pytestmark = pytest.mark.gpu


def residuals_dev(Td, Z):
    """rho_j = ||T z_j - lambda_j z_j||_2 / (||T||_F ||z_j||_2) on the GPU, with
    z_j rescaled to max |z| = 1 so that nothing overflows."""
    Tu = torch.triu(Td)
    lam = torch.diagonal(Tu)
    zs = Z / Z.abs().amax(dim=0, keepdim=True)
    R = Tu @ zs - zs * lam[None, :]
    return (torch.linalg.norm(R, dim=0) / (torch.linalg.norm(Tu) * torch.linalg.norm(zs, dim=0)))


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(1, 32), (2, 16), (97, 16), (300, 32), (640, 64), (1000, 32)])
def test_trevc_matches_oracle(m, nb, tensor):
    T = W.trevc_problem(m, seed=m + 1)
    Td = to_dev(T)
    Z, sc, se, st = msts.msts_trevc(Td, nb=nb, tensor=tensor)
    Zo, eo, sco = oracle.trevc(T, nb)
    eg = to_np(se)
    assert np.array_equal(eg, eo)
    assert np.array_equal(to_np(sc), sco)
    Zg = to_np(Z)
    assert (np.tril(Zg, -1) == 0).all()
    assert np.array_equal(np.diag(Zg).real, sco)
    scale = np.maximum(np.abs(Zo).max(axis=0), 1e-300)
    assert (np.abs(Zg - Zo).max(axis=0) / scale).max() <= 1e-8
    assert residuals_dev(Td, Z).max().item() <= 2 * m * EPS
    if m >= 640:
        assert eo.max() > 0 and int(st.item()) & 8


@pytest.mark.parametrize("tensor", [False, True])
def test_trevc_full_size_sampled_columns_and_residual(tensor):
    """Workload 2 at full size (4096 x 4096, clustered eigenvalues), in the launch
    configuration bench.py times: every column's eigen-residual on the GPU, and 12
    sampled columns against the oracle."""
    T = W.trevc_problem()
    Td = to_dev(T)
    Z, sc, se, st = msts.msts_trevc(Td, nb=32, tensor=tensor)
    rho = residuals_dev(Td, Z)
    assert rho.max().item() <= 2 * 4096 * EPS
    cols = [0, 1, 31, 32, 33, 1000, 2047, 2048, 3000, 4063, 4064, 4095]
    Zc, ec = oracle.trevc_columns(T, cols, 32)
    eg = to_np(se)[cols]
    Zg = to_np(Z[:, cols])
    assert np.array_equal(eg, ec)
    scale = np.maximum(np.abs(Zc).max(axis=0), 1e-300)
    assert (np.abs(Zg - Zc).max(axis=0) / scale).max() <= 1e-8
    assert to_np(se).max() > 0                      # scaling exercised
