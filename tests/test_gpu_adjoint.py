"""GPU parity: the adjoint (dL/dU, dL/dB, dL/ds) against the oracle gradient,
finite differences and the autograd Function."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("m,n,nb", [(64, 8, 32), (37, 5, 16), (200, 32, 64), (1, 1, 32)])
def test_adjoint_matches_oracle(m, n, nb):
    U, s, B = W.plain_problem(m, n, seed=4000 + m)
    g = W.rng(0, m)
    G = W.cn(g, (m, n))
    dU, dB, ds, st = msts.msts_adjoint(to_dev(U), to_dev(s), to_dev(B), to_dev(G), nb=nb)
    rU, rB, rs = oracle.adjoint(U, s, B, G)
    assert rel(to_np(dU), rU) <= 1e-9 and rel(to_np(dB), rB) <= 1e-9 and rel(to_np(ds), rs) <= 1e-9
    assert (np.tril(to_np(dU), -1) == 0).all()


@pytest.mark.parametrize("tensor", [False, True])
def test_adjoint_batched_uneven(tensor):
    probs = W.batch_problem(batch=5, m_lo=30, m_hi=120, n=7, seed=3)
    g = W.rng(0, 1)
    items = [(U, s, B, W.cn(g, B.shape)) for U, s, B in probs]
    outs, st = msts.msts_adjoint_batched([tuple(to_dev(a) for a in it) for it in items], nb=32, tensor=tensor)
    for (U, s, B, G), (dU, dB, ds) in zip(items, outs):
        rU, rB, rs = oracle.adjoint(U, s, B, G)
        assert rel(to_np(dU), rU) <= 1e-9 and rel(to_np(dB), rB) <= 1e-9 and rel(to_np(ds), rs) <= 1e-9


def test_autograd_function_central_differences():
    """loss = sum |x|^2 through MultiShiftSolve: backward vs central differences
    at h = 1e-6 on random directions (rel. err <= 1e-6)."""
    m, n = 96, 8
    U, s, B = W.plain_problem(m, n, seed=12)
    Ud = to_dev(U).requires_grad_()
    sd = to_dev(s).requires_grad_()
    Bd = to_dev(B).requires_grad_()
    X = msts.multishift_solve(Ud, sd, Bd)
    (X.abs() ** 2).sum().backward()
    gU, gs, gB = Ud.grad, sd.grad, Bd.grad

    def loss(U_, s_, B_):
        X_ = to_dev(B_)
        msts.msts_solve(to_dev(U_), to_dev(s_), X_, nb=32)
        return float((X_.abs() ** 2).sum())

    r = W.rng(0, 5)
    h = 1e-6
    for part in (1.0, 1j):
        EU = np.asfortranarray(np.triu(r.standard_normal((m, m))) * part)
        EB = np.asfortranarray(r.standard_normal((m, n)) * part)
        Es = r.standard_normal(n) * part
        fd = (loss(U + h * EU, s + h * Es, B + h * EB) - loss(U - h * EU, s - h * Es, B - h * EB)) / (2 * h)
        an = (np.vdot(to_np(gU), EU) + np.vdot(to_np(gB), EB) + np.vdot(to_np(gs), Es)).real
        assert abs(fd - an) <= 1e-6 * abs(an)
    rU, rB, rs = oracle.adjoint(U, s, B, 2 * oracle.solve(U, s, B))
    assert rel(to_np(gU), rU) <= 1e-9 and rel(to_np(gB), rB) <= 1e-9 and rel(to_np(gs), rs) <= 1e-9
