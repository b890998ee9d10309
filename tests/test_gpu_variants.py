"""GPU parity of the other triangular variants (footnote to Sec. 2: lower,
transposed and right-hand cases), plain and safe, both substitution-GEMM
paths, against the oracle; plus the exact reductions that the mapping onto
the upper-triangular engine must preserve bit for bit."""
import itertools

import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import EPS, to_dev, to_np

pytestmark = pytest.mark.gpu

VARIANTS = list(itertools.product(["left", "right"], ["upper", "lower"], ["N", "T", "C"]))


def tri(A, uplo):
    return np.triu(A) if uplo == "upper" else np.tril(A)


def op(A, trans):
    return A if trans == "N" else (A.T if trans == "T" else A.conj().T)


def problem(m, n, side, uplo, seed, junk=True):
    """Random triangle (off-diagonal CN/sqrt(m), unit-disk diagonal) with
    large junk in the other triangle, which must never be read."""
    g = W.rng(0, seed)
    A = W.cn(g, (m, m)) / np.sqrt(m)
    A[np.arange(m), np.arange(m)] = W.disk(g, m, 1.0)
    other = (np.tril(W.cn(g, (m, m)), -1) if uplo == "upper" else np.triu(W.cn(g, (m, m)), 1)) * 1e6
    A = np.asfortranarray(tri(A, uplo) + (other if junk else 0))
    s = W.separated_shifts(g, n, 1.5, np.diag(A), 0.05)
    B = np.asfortranarray(W.cn(g, (m, n) if side == "left" else (n, m)))
    return A, s, B


def forward_bound(A, s, uplo, trans, side, X, Xo, c=16.0):
    m = A.shape[0]
    n = s.size
    for j in range(n):
        M = op(tri(A, uplo), trans) - s[j] * np.eye(m)
        if side == "right":
            M = M.T
        kappa = np.linalg.norm(M, np.inf) * np.linalg.norm(np.linalg.inv(M), np.inf)
        x, xo = (X[:, j], Xo[:, j]) if side == "left" else (X[j, :], Xo[j, :])
        err = np.abs(x - xo).max() / np.abs(xo).max()
        assert err <= min(c * m * EPS * kappa, 1e-6), (j, err, kappa)


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_plain_variant_matches_oracle(side, uplo, trans, tensor):
    m, n, nb = 150, 21, 32
    A, s, B = problem(m, n, side, uplo, seed=900 + 7 * len(side) + len(uplo) + ord(trans))
    X = to_dev(B)
    _, _, _, st = msts.msts_solve_variant(to_dev(A), to_dev(s), X, side=side, uplo=uplo, trans=trans, nb=nb,
                                          tensor=tensor)
    assert int(st.item()) == 0
    forward_bound(A, s, uplo, trans, side, to_np(X), oracle.solve_variant(A, s, B, side, uplo, trans))


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
def test_safe_variant_exponents_equal_oracle_on_rescaling_problem(side, uplo, trans, tensor):
    """A clustered, badly scaled triangle (the TREVC workload's shape) with
    shifts 1e-9 from its eigenvalues: every variant rescales, and its scale
    exponents must equal the oracle's (Alg. 5 in the variant's order)."""
    m, n, nb = 256, 24, 32
    T = W.trevc_problem(m, seed=61, cluster_frac=0.1, offdiag_scale=30.0)
    A = np.asfortranarray(T if uplo == "upper" else T.T)
    g = W.rng(0, 62)
    s = np.diag(T)[g.permutation(m)[:n]] * (1 + 1e-9)
    if trans == "C":
        s = s.conj()                                  # eigenvalues of A^H are conj(diag)
    B = np.asfortranarray(W.cn(g, (m, n) if side == "left" else (n, m)))
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve_variant(to_dev(A), to_dev(s), X, side=side, uplo=uplo, trans=trans, nb=nb,
                                            safe=True, tensor=tensor)
    Xo, eo = oracle.safe_solve_variant(A, s, B, nb, side, uplo, trans)
    eg = to_np(se)
    assert eo.max() > 0
    assert np.array_equal(eg, eo)
    assert np.array_equal(to_np(sc), np.ldexp(1.0, -eo.astype(np.int64)))
    Xg = to_np(X)
    ax = 0 if side == "left" else 1
    rel = np.abs(Xg - Xo).max(axis=ax) / np.abs(Xo).max(axis=ax)
    assert rel.max() <= 1e-8


@pytest.mark.parametrize("side,uplo,trans", VARIANTS)
@pytest.mark.parametrize("m,n,nb", [(1, 1, 32), (37, 5, 16), (97, 40, 64)])
def test_safe_variant_ragged_sizes_match_oracle(side, uplo, trans, m, n, nb):
    A, s, B = problem(m, n, side, uplo, seed=950 + m)
    X = to_dev(B)
    _, _, se, _ = msts.msts_solve_variant(to_dev(A), to_dev(s), X, side=side, uplo=uplo, trans=trans, nb=nb,
                                          safe=True)
    Xo, eo = oracle.safe_solve_variant(A, s, B, nb, side, uplo, trans)
    assert np.array_equal(to_np(se), eo)
    forward_bound(A, s, uplo, trans, side, to_np(X), Xo)


@pytest.mark.parametrize("safe", [False, True])
def test_left_lower_is_the_reversed_upper_gpu_solve_bitwise(safe):
    """The lower solve runs the upper engine on J L J: bitwise equal to
    msts_solve called on the reversal built on the host."""
    m, n, nb = 300, 33, 32
    L, s, B = problem(m, n, "left", "lower", seed=970, junk=False)
    X1 = to_dev(B)
    _, _, e1, _ = msts.msts_solve_variant(to_dev(L), to_dev(s), X1, side="left", uplo="lower", trans="N", nb=nb,
                                          safe=safe)
    X2 = to_dev(np.asfortranarray(B[::-1, :]))
    _, _, e2, _ = msts.msts_solve(to_dev(np.asfortranarray(L[::-1, ::-1])), to_dev(s), X2, nb=nb, safe=safe)
    assert torch.equal(X1, torch.flip(X2, dims=[0]))
    if safe:
        assert torch.equal(e1, e2)


def test_right_upper_t_is_the_upper_solve_on_rows_bitwise():
    m, n, nb = 200, 17, 32
    U, s, B = problem(m, n, "right", "upper", seed=971, junk=False)
    X1 = to_dev(B)
    msts.msts_solve_variant(to_dev(U), to_dev(s), X1, side="right", uplo="upper", trans="T", nb=nb)
    X2 = to_dev(np.asfortranarray(B.T))
    msts.msts_solve(to_dev(U), to_dev(s), X2, nb=nb)
    assert torch.equal(X1, X2.T)


def test_left_upper_n_is_msts_solve_bitwise():
    U, s, B = W.plain_problem(256, 64, seed=972)
    X1, X2 = to_dev(B), to_dev(B)
    msts.msts_solve_variant(to_dev(U), to_dev(s), X1, nb=32, tensor=True)
    msts.msts_solve(to_dev(U), to_dev(s), X2, nb=32, tensor=True)
    assert torch.equal(X1, X2)


def test_scaling_study_size_lower_safe_sampled():
    """m = 4096, n = 512 (the scaling study's matrix shape: the upper triangle
    of a Hermitian matrix with eigenvalues in [1, 2], shifts in the disk
    B(1.5, 0.5)), read as its conjugate transpose: the left lower solve with
    the safe tensor-core path; 16 sampled columns against the oracle, and the
    normwise backward error of every column."""
    m, n, nb = 4096, 512, 32
    U, s, B = W.scaling_problem(m, n)
    L = np.asfortranarray(U.conj().T)
    Ld = to_dev(L)
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve_variant(Ld, to_dev(s), X, side="left", uplo="lower", trans="N", nb=nb,
                                            safe=True, tensor=True)
    cols = np.arange(0, n, 32)
    Xo, eo = oracle.safe_solve_variant(L, s[cols], B[:, cols], nb, "left", "lower", "N")
    assert np.array_equal(to_np(se)[cols], eo)
    Xg = to_np(X)
    rel = np.abs(Xg[:, cols] - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8
    Lt = torch.tril(Ld)
    sd = to_dev(s)
    Bd = to_dev(B)
    R = Lt @ X - X * sd[None, :] - Bd * sc[None, :]
    nrmM = (Lt.abs().sum(dim=1).max() + sd.abs()).max()
    eta = R.abs().amax(dim=0) / (nrmM * X.abs().amax(dim=0) + sc * Bd.abs().amax(dim=0))
    assert eta.max().item() <= 8 * m * EPS
