"""GPU edge cases of every entry point: empty problems (m = 0 or n = 0) are
no-ops that launch nothing and leave the outputs alone, zero right-hand
sides solve to zero with unit scales, and exact zero pivots are flagged (plain)
or replaced by delta (safe), as the oracle does."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def zeros(rows, cols):
    return msts.colmajor(torch.zeros((rows, cols), dtype=torch.complex128, device="cuda"))


def cvec(n):
    return torch.zeros(n, dtype=torch.complex128, device="cuda")


@pytest.mark.parametrize("safe", [False, True])
@pytest.mark.parametrize("tensor", [False, True])
def test_empty_solves_launch_nothing(safe, tensor):
    lib = msts.load_library()
    U = to_dev(W.plain_problem(40, 3, seed=1)[0])
    before = lib.msts_launch_count()
    B = zeros(40, 0)
    _, sc, se, st = msts.msts_solve(U, cvec(0), B, safe=safe, tensor=tensor)
    B0 = zeros(0, 5)
    msts.msts_solve(zeros(0, 0), cvec(5), B0, safe=safe, tensor=tensor)
    msts.msts_gsolve(U, U, cvec(0), zeros(40, 0), safe=safe, tensor=tensor)
    msts.msts_solve_variant(U, cvec(0), zeros(0, 40), side="right", uplo="lower", trans="C", safe=safe,
                            tensor=tensor)
    msts.msts_solve_variant(zeros(0, 0), cvec(3), zeros(0, 3), side="left", uplo="lower", safe=safe,
                            tensor=tensor)
    est, kind, steps, _ = msts.msts_pseudospectra_1norm(U, cvec(0), tensor=tensor)
    torch.cuda.synchronize()
    assert lib.msts_launch_count() == before
    assert est.numel() == 0 and int(st.item()) == 0


def test_empty_trevc_and_back_transform():
    lib = msts.load_library()
    before = lib.msts_launch_count()
    Z, sc, se, st = msts.msts_trevc(zeros(0, 0))
    X, st2 = msts.msts_back_transform(zeros(0, 0), zeros(0, 0))
    torch.cuda.synchronize()
    assert Z.numel() == 0 and X.numel() == 0 and lib.msts_launch_count() == before


@pytest.mark.parametrize("tensor", [False, True])
def test_zero_right_hand_sides(tensor):
    U, s, B = W.plain_problem(100, 7, seed=5)
    Bz = np.zeros_like(B)
    X = to_dev(Bz)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=32, tensor=tensor)
    assert (to_np(X) == 0).all() and (to_np(se) == 0).all() and (to_np(sc) == 1.0).all()
    assert int(st.item()) == 0


def test_plain_zero_pivot_is_flagged():
    U, s, B = W.plain_problem(64, 4, seed=6)
    s = s.copy()
    s[2] = U[10, 10]                                    # U(10,10) - s_2 = 0 exactly
    X = to_dev(B)
    _, _, _, st = msts.msts_solve(to_dev(U), to_dev(s), X, nb=32)
    assert int(st.item()) & 1                           # MSTS_STATUS_ZERO_PIVOT
    Xg = to_np(X)
    assert np.isfinite(Xg[:, [0, 1, 3]]).all()          # the other shifts are unaffected


@pytest.mark.parametrize("tensor", [False, True])
def test_safe_zero_pivot_uses_delta_like_the_oracle(tensor):
    U, s, B = W.plain_problem(64, 4, seed=7)
    s = s.copy()
    s[1] = U[20, 20]
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=32, tensor=tensor)
    Xo, eo = oracle.safe_solve(U, s, B, 32)
    assert int(st.item()) & 16                          # MSTS_STATUS_DELTA
    assert np.array_equal(to_np(se), eo)
    Xg = to_np(X)
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8


def _rescale_fixture(m):
    """The 2x2 safe-solve fixture of tests/golden (U(0,0) = 1, U(0,m-1) = -5,
    U(m-1,m-1) = 3, b = 3*2^958 e_{m-1}), embedded in an m x m identity so that
    with n_b < m the rescale comes from Alg. 5's block bound C_blk = 5."""
    U = np.eye(m, dtype=np.complex128)
    U[0, m - 1] = -5.0
    U[m - 1, m - 1] = 3.0
    B = np.zeros((m, 1), dtype=np.complex128)
    B[m - 1, 0] = np.ldexp(3.0, 958)
    x = np.zeros(m, dtype=np.complex128)
    x[0], x[m - 1] = np.ldexp(5.0, 956), np.ldexp(1.0, 956)
    return np.asfortranarray(U), np.asfortranarray(B), x


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(2, 32), (33, 32), (17, 16)])
def test_safe_rescale_exponent_fixture(m, nb, tensor):
    """The exact rescale exponent of Alg. 4 / Alg. 5 (smallest k with
    2^-k G < Omega; here G = 2^961, so k = 2): the GPU's scale exponent equals
    the hand-derived one and the oracle's, and x is the exact solution times 2^-2."""
    U, B, x = _rescale_fixture(m)
    s = np.zeros(1, dtype=np.complex128)
    Xd = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), Xd, safe=True, nb=nb, tensor=tensor)
    Xo, eo = oracle.safe_solve(U, s, B, nb)
    assert int(to_np(se)[0]) == 2 == int(eo[0])
    assert to_np(sc)[0] == 0.25
    X = to_np(Xd)[:, 0]
    assert np.abs(X - x).max() <= 4 * np.finfo(float).eps * np.abs(x).max()


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(2, 32), (33, 32), (17, 16)])
def test_safe_gsolve_rescale_exponent_fixture(m, nb, tensor):
    """The generalized form of the fixture above (Alg. 9): U = 2I with
    U(m-1,m-1) = 4 and V = I + 5 e_0 e_{m-1}^T, lambda = 1, so that U - lambda V
    is the matrix above with its off-diagonal growth coming from V alone;
    e = 2 exactly and x exact on both GEMM paths."""
    Ustd, B, x = _rescale_fixture(m)
    U = 2.0 * np.eye(m, dtype=np.complex128)
    U[m - 1, m - 1] = 4.0
    V = np.eye(m, dtype=np.complex128)
    V[0, m - 1] = 5.0
    U, V = np.asfortranarray(U), np.asfortranarray(V)
    assert np.array_equal(U - V, Ustd)
    lam = np.ones(1, dtype=np.complex128)
    Xd = to_dev(B)
    _, sc, se, st = msts.msts_gsolve(to_dev(U), to_dev(V), to_dev(lam), Xd, safe=True, nb=nb, tensor=tensor)
    Xo, eo = oracle.safe_gsolve(U, V, lam, B, nb)
    assert int(to_np(se)[0]) == 2 == int(eo[0])
    assert to_np(sc)[0] == 0.25
    X = to_np(Xd)[:, 0]
    assert np.abs(X - x).max() <= 4 * np.finfo(float).eps * np.abs(x).max()
