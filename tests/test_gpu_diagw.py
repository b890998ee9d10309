"""GPU parity of the four-warp layout of the diagonal-block step (n_b = 32).

Every value sees the same operations in the same order whatever the layout, so
the four-warp layout with 1, 2 or 4 lanes per shift and the one-warp layout
must give the same results bit for bit (X, scale factors and exponents, and
the digit planes the tensor-core step consumes), on plain, safe (rescaling)
and conjugate-transposed solves and on TREVC's shortcut; blocks that take the
serial safeguarded loop still match the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

LAYOUTS = (-1, 1, 2, 4)      # one-warp layout, then four-warp with 1, 2, 4 lanes per shift


def with_layout(value, fn):
    lib = msts.load_library()
    assert lib.msts_tune_set(1, value) == 0
    try:
        out = fn()
        torch.cuda.synchronize()
        return out
    finally:
        assert lib.msts_tune_set(1, 0) == 0


def rescaling_problem(m, n, seed):
    """Shifts next to eigenvalues and off-diagonal entries large enough (for
    the order m) that every column rescales."""
    scale = 30.0 if m >= 200 else (1000.0 if m >= 96 else 1e5)
    T = W.trevc_problem(m, seed=seed, cluster_frac=0.1, offdiag_scale=scale)
    g = W.rng(0, seed + 3)
    B = W.cn(g, (m, n))
    shifts = np.diag(T)[g.integers(0, m, n)] + 1e-9
    return T, shifts, B


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("kind", ["plain", "safe", "conj"])
@pytest.mark.parametrize("m,n", [(300, 40), (97, 5), (64, 70)])
def test_every_layout_gives_the_same_bits(kind, tensor, m, n):
    if kind == "safe":
        U, s, B = rescaling_problem(m, n, 700 + m)
    else:
        U, s, B = W.plain_problem(m, n, seed=800 + m)
    Ud, sd = to_dev(U), to_dev(s)
    res = []
    for lay in LAYOUTS:
        X = to_dev(B)
        _, sc, se, st = with_layout(lay, lambda: msts.msts_solve(Ud, sd, X, safe=kind == "safe",
                                                                 conj_trans=kind == "conj", nb=32, tensor=tensor))
        res.append((X, sc, se, int(st.item())))
    X0, sc0, se0, st0 = res[0]
    for X, sc, se, st in res[1:]:
        assert torch.equal(X, X0) and st == st0
        if kind == "safe":
            assert torch.equal(sc, sc0) and torch.equal(se, se0)
    if kind == "safe":
        Xo, eo = oracle.safe_solve(U, s, B, 32)
        assert np.array_equal(to_np(se0), eo) and eo.max() > 0
        rel = np.abs(to_np(X0) - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
        assert rel.max() <= 1e-8
    else:
        Xo = oracle.solve(U, s, B, conj_trans=kind == "conj")
        rel = np.abs(to_np(X0) - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
        assert rel.max() <= 1e-9


@pytest.mark.parametrize("tensor", [False, True])
def test_trevc_every_layout_gives_the_same_bits(tensor):
    """TREVC (strictly-upper shortcut: columns cut at row j inside a block)."""
    T = W.trevc_problem(330, seed=71)
    Td = to_dev(T)
    res = [with_layout(lay, lambda: msts.msts_trevc(Td, nb=32, tensor=tensor)) for lay in LAYOUTS]
    Z0, sc0, se0, _ = res[0]
    for Z, sc, se, _ in res[1:]:
        assert torch.equal(Z, Z0) and torch.equal(se, se0) and torch.equal(sc, sc0)
    Zo, eo, _ = oracle.trevc(T, 32)
    assert np.array_equal(to_np(se0), eo)


@pytest.mark.parametrize("lanes", [1, 2, 4])
def test_serial_fallback_in_the_four_warp_layout(lanes):
    """A subnormal pivot sends its CTA through the serial safeguarded loop (one
    thread per shift): exponents equal to the oracle's, X within 1e-8."""
    U, s, B = W.plain_problem(96, 40, seed=21)
    U[40, 40] = 1e-310
    s[2] = 0.0
    X = to_dev(B)
    _, sc, se, st = with_layout(lanes, lambda: msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=32))
    Xo, eo = oracle.safe_solve(U, s, B, 32)
    assert eo[2] > 0
    assert np.array_equal(to_np(se), eo)
    Xg = to_np(X)
    assert np.isfinite(Xg).all()
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8


def test_many_shifts_every_lane_width_same_bits():
    """Enough shifts for several CTAs per SM (4864 columns, m = 96)."""
    U, s, B = rescaling_problem(96, 4864, 905)
    Ud, sd = to_dev(U), to_dev(s)
    res = []
    for lay in (1, 2, 4, -1):
        X = to_dev(B)
        _, sc, se, _ = with_layout(lay, lambda: msts.msts_solve(Ud, sd, X, safe=True, nb=32, tensor=True))
        res.append((X, se))
    for X, se in res[1:]:
        assert torch.equal(X, res[0][0]) and torch.equal(se, res[0][1])
