"""Helpers for the GPU parity tests (numpy <-> column-major CUDA tensors)."""
import numpy as np
import torch

import paper_1607_01477_gb300 as msts

EPS = np.finfo(np.float64).eps


def dev():
    return torch.device("cuda:0")


def to_dev(a):
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev())
    return msts.colmajor(torch.from_numpy(np.asfortranarray(a)).to(dev()))


def to_np(t):
    t = t.detach().cpu()
    if t.dim() == 2:
        return np.asfortranarray(t.numpy())
    return t.numpy()


def cond_inf(U, shifts):
    """kappa_inf(U - s_j I) for every shift (numpy, small m only)."""
    Ut = np.triu(U)
    m = Ut.shape[0]
    out = []
    for s in shifts:
        A = Ut - s * np.eye(m)
        out.append(np.linalg.norm(A, np.inf) * np.linalg.norm(np.linalg.inv(A), np.inf))
    return np.array(out)


def forward_close(X, Xo, kappa, m, c=16.0):
    """Per-column forward difference bound for two backward-stable solvers:
    ||x - x_o||_inf <= c m eps kappa_j ||x_o||_inf (and never looser than 1e-6)."""
    tol = np.minimum(c * m * EPS * kappa, 1e-6)
    err = np.abs(X - Xo).max(axis=0) / np.maximum(np.abs(Xo).max(axis=0), 1e-300)
    return err, tol
