"""GPU: the tensor-core FP64-accurate residual (BF16 digit planes on tcgen05)
against the FP64 FMA residual and, for exactly representable inputs, bit for bit."""
import numpy as np
import pytest
import torch

import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def int_problem(m, n, seed, scale_u=1.0, scale_x=1.0):
    """Small-integer entries times powers of two: every product and partial sum is
    exact in FP64 and in the digit planes, so both residuals must agree bitwise."""
    g = np.random.default_rng(seed)
    U = np.triu(g.integers(-60, 61, (m, m)) + 1j * g.integers(-60, 61, (m, m))) * scale_u
    X = (g.integers(-90, 91, (m, n)) + 1j * g.integers(-90, 91, (m, n))) * scale_x
    B = g.integers(-9, 10, (m, n)) + 1j * g.integers(-9, 10, (m, n))
    s = (g.integers(-5, 6, n) + 1j * g.integers(-5, 6, n)).astype(np.complex128)
    return (np.asfortranarray(U.astype(np.complex128)), s, np.asfortranarray(B.astype(np.complex128)),
            np.asfortranarray(X.astype(np.complex128)))


@pytest.mark.parametrize("m,n", [(64, 32), (100, 45), (300, 64), (513, 97)])
def test_ozaki_residual_bitwise_on_exact_inputs(m, n):
    U, s, B, X = int_problem(m, n, seed=m + n, scale_u=2.0 ** -3, scale_x=2.0 ** 5)
    Ud, sd, Bd, Xd = to_dev(U), to_dev(s), to_dev(B), to_dev(X)
    R64, st64 = msts.msts_residual(Ud, sd, Bd, Xd)
    Roz, stoz = msts.msts_residual(Ud, sd, Bd, Xd, ozaki=True)
    assert int(stoz.item()) == 0
    ref = B - (np.triu(U) @ X - X * s[None, :])
    assert np.array_equal(to_np(R64), ref)
    assert np.array_equal(to_np(Roz), ref)


@pytest.mark.parametrize("m,n", [(64, 32), (200, 70), (1000, 100)])
def test_ozaki_residual_matches_fp64(m, n):
    """Random FP64 data: agreement to the method's bound, 2^-48 K' max|U_r| max|X_j|."""
    U, s, B = W.mixed_problem(m, n, seed=m)
    X = np.asfortranarray(W.cn(W.rng(0, m), (m, n)))
    Ud, sd, Bd, Xd = to_dev(U), to_dev(s), to_dev(B), to_dev(X)
    R64, _ = msts.msts_residual(Ud, sd, Bd, Xd)
    Roz, st = msts.msts_residual(Ud, sd, Bd, Xd, ozaki=True)
    assert int(st.item()) == 0
    d = np.abs(to_np(Roz) - to_np(R64))
    ur = np.maximum(np.abs(np.triu(U).real), np.abs(np.triu(U).imag)).max(axis=1)
    xc = np.maximum(np.abs(X.real), np.abs(X.imag)).max(axis=0)
    bound = 2.0 ** -48 * (2 * m) * ur[:, None] * xc[None, :] * 4
    assert (d <= bound).all(), (d / bound).max()


def test_mixed_with_ozaki_residual_reaches_target():
    U, s, B = W.mixed_problem(700, 96, seed=4)
    X, info, st = msts.msts_solve_mixed(to_dev(U), to_dev(s), to_dev(B), tol=1e-12,
                                        flags=msts.MSTS_RESIDUAL_OZAKI)
    assert info["eta"] <= 1e-12 and int(st.item()) == 0
    Xf, info_f, _ = msts.msts_solve_mixed(to_dev(U), to_dev(s), to_dev(B), tol=1e-12)
    rel = (np.abs(to_np(X) - to_np(Xf)).max(axis=0) / np.abs(to_np(Xf)).max(axis=0)).max()
    assert rel <= 1e-11
