"""GPU parity: the mixed-precision solve with FP64 iterative refinement against
the FP64 oracle (relative residual <= 1e-12 after refinement)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from conftest import backward_error
from gpu_util import EPS, cond_inf, forward_close, to_dev, to_np

pytestmark = pytest.mark.gpu


FP32_GEMM, OZ = msts.MSTS_MIXED_FP32_GEMM, msts.MSTS_RESIDUAL_OZAKI


@pytest.mark.parametrize("flags", [0, FP32_GEMM, OZ, OZ | FP32_GEMM])
@pytest.mark.parametrize("m,n,nb", [(300, 40, 32), (129, 7, 16), (64, 64, 64), (1, 3, 32), (600, 40, 32)])
def test_mixed_matches_oracle(m, n, nb, flags):
    """Both low-precision products (the tensor cores' 3-plane split-BF16 one by
    default, FP32 FMA on request) with both residuals (FP64 FMA, tensor-core
    digit planes) reach eta <= 1e-12 and the oracle's solution."""
    U, s, B = W.mixed_problem(m, n, seed=500 + m)
    X, info, st = msts.msts_solve_mixed(to_dev(U), to_dev(s), to_dev(B), tol=1e-12, nb=nb, flags=flags)
    Xg = to_np(X)
    assert info["eta"] <= 1e-12
    assert info["eta_before"] > info["eta"] or info["eta_before"] <= 1e-12
    eta = backward_error(U, s, Xg, B)
    assert eta.max() <= 1e-12
    Xo = oracle.solve(U, s, B)
    err, tol = forward_close(Xg, Xo, cond_inf(U, s), m, c=64.0)
    assert (err <= np.maximum(tol, 1e-11)).all()
    assert int(st.item()) == 0


@pytest.mark.parametrize("flags", [0, FP32_GEMM])
def test_mixed_first_solve_is_low_precision(flags):
    """Before refinement the low-precision solve is far from FP64 (the 3-plane
    tensor-core product and the FP32 product alike: eta ~ 1e-7); one to three
    corrections reach the 1e-12 target."""
    U, s, B = W.mixed_problem(512, 32, seed=9)
    X, info, st = msts.msts_solve_mixed(to_dev(U), to_dev(s), to_dev(B), tol=1e-12, flags=flags)
    assert 1e-10 < info["eta_before"] < 1e-4
    assert 1 <= info["iters"] <= 3


def test_mixed_cap_reports_not_converged():
    U, s, B = W.mixed_problem(200, 8, seed=2)
    X, info, st = msts.msts_solve_mixed(to_dev(U), to_dev(s), to_dev(B), tol=0.0, max_iter=1)
    assert info["iters"] == 1
    assert int(st.item()) & 32                      # MSTS_STATUS_NOT_CONVERGED


def test_mixed_full_size_sampled_columns():
    """Workload 3 at full size (8192 x 8192, 2048 shifts): the library's eta is
    re-checked on the GPU for every column with an independent complex128
    product, and 6 sampled columns are compared with the oracle."""
    U, s, B = W.mixed_problem()
    Ud, sd, Bd = to_dev(U), to_dev(s), to_dev(B)
    X, info, st = msts.msts_solve_mixed(Ud, sd, Bd, tol=1e-12, flags=OZ)
    assert info["eta"] <= 1e-12 and 1e-10 < info["eta_before"] < 1e-4
    Ut = torch.triu(Ud)
    R = Bd - (Ut @ X - X * sd[None, :])
    rown = Ut.abs().sum(dim=1) - torch.diagonal(Ut).abs()
    anorm = (rown[:, None] + (torch.diagonal(Ut)[:, None] - sd[None, :]).abs()).amax(dim=0)
    eta = R.abs().amax(dim=0) / (anorm * X.abs().amax(dim=0) + Bd.abs().amax(dim=0))
    assert eta.max().item() <= 1e-12
    cols = [0, 1, 777, 1024, 2000, 2047]
    Xo = oracle.solve(U, s[cols], np.asfortranarray(B[:, cols]))
    Xg = to_np(X[:, cols])
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-9
