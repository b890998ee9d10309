import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


EPS = np.finfo(np.float64).eps


def backward_error(U, shifts, X, B, scales=None, conj_trans=False):
    """Per-column normwise backward error
    eta_j = ||(A_j) x_j - s_j b_j||_inf / (||A_j||_inf ||x_j||_inf + s_j ||b_j||_inf),
    A_j = U - s_j I (or U^H - conj(s_j) I), computed in numpy (a check, not the oracle)."""
    Ut = np.triu(U)
    if conj_trans:
        Ut = Ut.conj().T
        sh = np.conj(shifts)
    else:
        sh = shifts
    m, n = X.shape
    sc = np.ones(n) if scales is None else scales
    etas = np.empty(n)
    rowabs = np.abs(Ut).sum(axis=1)
    for j in range(n):
        A_x = Ut @ X[:, j] - sh[j] * X[:, j]
        r = A_x - sc[j] * B[:, j]
        anorm = np.max(rowabs - np.abs(np.diag(Ut)) + np.abs(np.diag(Ut) - sh[j]))
        den = anorm * np.abs(X[:, j]).max() + sc[j] * np.abs(B[:, j]).max()
        etas[j] = np.abs(r).max() / den if den > 0 else 0.0
    return etas
