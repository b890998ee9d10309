"""Pins for the oracle's adjoint: gradients of a real loss through
X = (U - s_j I)^{-1} b_j, checked against torch CPU autograd and finite differences."""
import numpy as np
import pytest
import torch

import oracle
from paper_1607_01477_gb300 import workloads as W


def torch_grads(U, s, B):
    """Independent gradient: autograd through dense per-shift torch.linalg.solve
    on the CPU, loss = sum |x|^2 (so G_X = 2X)."""
    Ut = torch.tensor(np.triu(U), requires_grad=True)
    st = torch.tensor(s, requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    m = U.shape[0]
    eye = torch.eye(m, dtype=torch.complex128)
    Ufull = torch.triu(Ut)
    loss = 0
    for j in range(B.shape[1]):
        x = torch.linalg.solve(Ufull - st[j] * eye, Bt[:, j])
        loss = loss + (x.abs() ** 2).sum()
    loss.backward()
    return torch.triu(Ut.grad).numpy(), Bt.grad.numpy(), st.grad.numpy()


@pytest.mark.parametrize("m,n", [(1, 1), (9, 3), (40, 6)])
def test_adjoint_matches_torch_autograd(m, n):
    U, s, B = W.plain_problem(m, n, seed=300 + m)
    X = oracle.solve(U, s, B)
    dU, dB, ds = oracle.adjoint(U, s, B, 2 * X)
    rU, rB, rs = torch_grads(U, s, B)
    for a, b in ((dU, rU), (dB, rB), (ds, rs)):
        assert np.abs(a - b).max() <= 1e-10 * max(1.0, np.abs(b).max())
    assert (np.tril(dU, -1) == 0).all()


def test_adjoint_central_differences():
    """Central differences at h = 1e-6 on random real and imaginary directions."""
    m, n = 30, 4
    U, s, B = W.plain_problem(m, n, seed=17)
    loss = lambda U_, s_, B_: float((np.abs(oracle.solve(U_, s_, B_)) ** 2).sum())
    X = oracle.solve(U, s, B)
    dU, dB, ds = oracle.adjoint(U, s, B, 2 * X)
    g = W.rng(0, 99)
    h = 1e-6
    for _ in range(3):
        for part in (1.0, 1j):
            EU = np.asfortranarray(np.triu(g.standard_normal((m, m))) * part)
            EB = np.asfortranarray(g.standard_normal((m, n)) * part)
            Es = g.standard_normal(n) * part
            fd = (loss(U + h * EU, s + h * Es, B + h * EB) - loss(U - h * EU, s - h * Es, B - h * EB)) / (2 * h)
            an = (np.vdot(dU, EU) + np.vdot(dB, EB) + np.vdot(ds, Es)).real
            assert abs(fd - an) <= 1e-6 * abs(an)


def test_adjoint_diagonal_closed_form():
    """Diagonal U: x = b/(d - s) and lambda = g / conj(d - s) in closed form; the
    upper-triangular gradient is -sum_j lambda_j(r) conj(x_j(c)) for r <= c."""
    g = W.rng(0, 12)
    m, n = 8, 3
    d = W.disk(g, m)
    U = np.asfortranarray(np.diag(d))
    s = W.disk(g, n, 1.5)
    B = W.cn(g, (m, n))
    G = W.cn(g, (m, n))
    dU, dB, ds = oracle.adjoint(U, s, B, G)
    X = B / (d[:, None] - s[None, :])
    L = G / np.conj(d[:, None] - s[None, :])
    assert np.allclose(dB, L, rtol=1e-13, atol=0)
    assert np.allclose(dU, np.triu(-(L @ X.conj().T)), rtol=1e-12, atol=1e-13)
    assert np.allclose(ds, (np.conj(X) * L).sum(axis=0), rtol=1e-12)


def test_adjoint_at_the_largest_batched_size():
    """A problem of the batched differentiable workload at its largest order
    (m = 2048, 32 shifts in the disk of radius 1.5): the oracle's gradients
    against CPU autograd through torch.linalg.solve_triangular (a library
    triangular solve per shift), and central differences (h = 1e-6) on random
    real and imaginary directions within 1e-6."""
    (U, s, B), = W.batch_problem(batch=1, m_lo=2048, m_hi=2048, seed=2048)
    m, n = B.shape
    X = oracle.solve(U, s, B)
    dU, dB, ds = oracle.adjoint(U, s, B, 2 * X)
    assert (np.tril(dU, -1) == 0).all()

    Ut = torch.tensor(np.triu(U), requires_grad=True)
    st = torch.tensor(s, requires_grad=True)
    Bt = torch.tensor(B, requires_grad=True)
    eye = torch.eye(m, dtype=torch.complex128)
    loss = 0
    for j in range(n):
        x = torch.linalg.solve_triangular(torch.triu(Ut) - st[j] * eye, Bt[:, j:j + 1], upper=True)
        loss = loss + (x.abs() ** 2).sum()
    loss.backward()
    for a, b in ((dU, torch.triu(Ut.grad).numpy()), (dB, Bt.grad.numpy()), (ds, st.grad.numpy())):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()

    f = lambda U_, s_, B_: float((np.abs(oracle.solve(U_, s_, B_)) ** 2).sum())
    g = W.rng(0, 2049)
    h = 1e-6
    for part in (1.0, 1j):
        EU = np.asfortranarray(np.triu(g.standard_normal((m, m))) * part)
        EB = np.asfortranarray(g.standard_normal((m, n)) * part)
        Es = g.standard_normal(n) * part
        fd = (f(U + h * EU, s + h * Es, B + h * EB) - f(U - h * EU, s - h * Es, B - h * EB)) / (2 * h)
        an = (np.vdot(dU, EU) + np.vdot(dB, EB) + np.vdot(ds, Es)).real
        assert abs(fd - an) <= 1e-6 * abs(an)
