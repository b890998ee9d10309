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


def colmajor_copy(t):
    return msts.colmajor(t.clone())


def _colrel(a, b):
    """Per column: max |a - b| over the column / max |b| over the column."""
    return (np.abs(a - b).max(axis=0) / np.maximum(np.abs(b).max(axis=0), 1e-300)).max()


def _blockrel(a, b, nb=32):
    """Per block of nb rows: max |a - b| over the rows / max |b| over the rows."""
    out = 0.0
    for r in range(0, b.shape[0], nb):
        den = np.abs(b[r:r + nb]).max()
        if den > 0:
            out = max(out, np.abs(a[r:r + nb] - b[r:r + nb]).max() / den)
    return out


@pytest.mark.parametrize("tensor", [False, True])
def test_adjoint_batched_full_workload_vs_oracle(tensor):
    """The whole differentiable batched workload (64 problems, m uniform in
    256..2048, 32 shifts each) in one batched adjoint call.  On the largest,
    the smallest and a middle problem, dB per column, dU per 32-row block and
    ds per shift (relative to ||x_j|| ||lambda_j||, which bounds |ds_j|) agree
    with the oracle within 1e-10; the tensor path exercises the batched
    digit-plane kernels at multi-tile, multi-chunk sizes (m up to 2034)."""
    probs = W.batch_problem()
    g = W.rng(0, 5005)
    items = [(U, s, B, W.cn(g, B.shape)) for U, s, B in probs]
    outs, st = msts.msts_adjoint_batched([tuple(to_dev(a) for a in it) for it in items], nb=32,
                                         tensor=tensor)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ms = np.array([U.shape[0] for U, _, _ in probs])
    order = np.argsort(ms)
    for i in (int(order[-1]), int(order[0]), int(order[len(order) // 2])):
        U, s, B, G = items[i]
        dU, dB, ds = (to_np(t) for t in outs[i])
        rU, rB, rs = oracle.adjoint(U, s, B, G)
        X = oracle.solve(U, s, B)
        assert _colrel(dB, rB) <= 1e-10, i
        assert _blockrel(dU, rU) <= 1e-10, i
        scale = np.linalg.norm(X, axis=0) * np.linalg.norm(rB, axis=0)
        assert (np.abs(ds - rs) / scale).max() <= 1e-10, i
        assert (np.tril(dU, -1) == 0).all()
    assert max(ms) >= 2000


@pytest.mark.parametrize("tensor", [False, True])
def test_adjoint_largest_batched_problem_central_differences(tensor):
    """L = sum |x|^2 on the largest problem of the batched workload: the GPU
    adjoint's directional derivative against central differences of GPU
    solves (h = 1e-6), two random directions for each of the real and the
    imaginary parts, relative error <= 1e-6."""
    probs = W.batch_problem()
    U, s, B = max(probs, key=lambda p: p[0].shape[0])
    m, n = B.shape
    Ud, sd, Bd = to_dev(U), to_dev(s), to_dev(B)
    X = to_dev(B)
    msts.msts_solve(Ud, sd, X, nb=32, tensor=tensor)
    outs, _ = msts.msts_adjoint_batched([(Ud, sd, Bd, colmajor_copy(2 * X))], nb=32, tensor=tensor)
    gU, gB, gs = (to_np(t) for t in outs[0])

    def loss(U_, s_, B_):
        X_ = to_dev(B_)
        msts.msts_solve(to_dev(U_), to_dev(s_), X_, nb=32, tensor=tensor)
        return float((X_.abs() ** 2).sum())

    r = W.rng(0, 2035)
    h = 1e-6
    for part in (1.0, 1.0, 1j, 1j):
        EU = np.asfortranarray(np.triu(r.standard_normal((m, m))) * part)
        EB = np.asfortranarray(r.standard_normal((m, n)) * part)
        Es = r.standard_normal(n) * part
        fd = (loss(U + h * EU, s + h * Es, B + h * EB) - loss(U - h * EU, s - h * Es, B - h * EB)) / (2 * h)
        an = (np.vdot(gU, EU) + np.vdot(gB, EB) + np.vdot(gs, Es)).real
        assert abs(fd - an) <= 1e-6 * abs(an)

