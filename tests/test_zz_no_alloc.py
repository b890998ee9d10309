"""The allocation-free safe solve (msts_safe_solve_static) against the regular
workspace entry point (msts_solve with MSTS_SAFE), through the C ABI.

The allocation-free form exists for callers that may not allocate device
memory when they need the solve (cudaMalloc synchronises the device and can
fail at run time); its scratch is a static device array shared by all calls.
This file is collected last so that a failure here never hides another test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MSTS_ERR_STATIC_SCRATCH = -1001


def _entry():
    lib = msts.load_library()
    f = lib.msts_safe_solve_static
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    f.restype = ctypes.c_int
    f.argtypes = [vp, i64, i64, vp, i64, vp, i64, vp, vp, ctypes.c_int32, vp, vp]
    return f


def _dev(a):
    a = np.asarray(a)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return msts.colmajor(torch.from_numpy(np.asfortranarray(a)).cuda())


def _solve_static(f, Td, sd, B, nb):
    """One call of the allocation-free entry point; returns (X, scales, exps, status)."""
    m, n = B.shape
    Xs = _dev(B)
    scs = torch.empty(n, dtype=torch.float64, device="cuda")
    ses = torch.empty(n, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = f(Td.data_ptr(), Td.stride(1), m, sd.data_ptr(), n, Xs.data_ptr(), m, scs.data_ptr(),
           ses.data_ptr(), nb, status.data_ptr(), stream)
    assert rc == 0
    return Xs, scs, ses, status


def _rescaling_problem(m, n, seed, exact_shift_rows=0):
    """Upper-triangular T with large off-diagonal entries and shifts next to
    its eigenvalues (so that Alg. 5 rescales); the first exact_shift_rows
    shifts equal diagonal entries exactly (zero pivots: the delta path)."""
    T = W.trevc_problem(m, seed=seed, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, seed + 1)
    B = W.cn(g, (m, n))
    d = np.diag(T)
    shifts = d[g.integers(0, m, n)] + 1e-9
    shifts[:exact_shift_rows] = d[g.integers(0, m, exact_shift_rows)]
    return T, shifts, B


def test_static_scratch_solve_matches_workspace_solve_bitwise():
    """Two calls in a row on different problems (the second smaller, with
    other shifts and with zero pivots, so that scratch left by the first call
    is never what the second needs): each equals msts_solve(MSTS_SAFE) on the
    same inputs bit for bit (the same deterministic kernels and launches), and
    the oracle's Alg. 5 on scale exponents (equal) and X (1e-8 per column)."""
    f = _entry()
    nb = 32
    for call, (m, n, seed, nzero) in enumerate([(300, 24, 44, 0), (200, 11, 71, 3)]):
        T, shifts, B = _rescaling_problem(m, n, seed, nzero)
        Td, sd = _dev(T), _dev(shifts)
        Xw = _dev(B)
        _, scw, sew, stw = msts.msts_solve(Td, sd, Xw, safe=True, nb=nb)
        Xs, scs, ses, st = _solve_static(f, Td, sd, B, nb)
        torch.cuda.synchronize()
        assert torch.equal(Xs, Xw) and torch.equal(scs, scw) and torch.equal(ses, sew), call
        assert int(st.item()) == int(stw.item())
        assert int(st.item()) & 8                       # MSTS_STATUS_SCALED
        assert bool(int(st.item()) & 16) == (nzero > 0) # MSTS_STATUS_DELTA
        Xo, eo = oracle.safe_solve(T, shifts, B, nb)
        assert np.array_equal(ses.cpu().numpy(), eo) and int(eo.max()) > 0
        x = Xs.cpu().numpy()
        rel = np.abs(x - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
        assert rel.max() <= 1e-8, call


def test_static_scratch_solve_just_under_the_limit():
    """A problem whose scratch is just under the 16 MiB array (m = 512 and the
    largest n that fits): bitwise equal to msts_solve(MSTS_SAFE), and 16
    sampled columns against the oracle (equal exponents, X within 1e-8)."""
    f = _entry()
    lib = msts.load_library()
    m, nb, limit = 512, 32, 16 << 20
    lo, hi = 1, 1 << 22
    while hi - lo > 1:                                  # largest n with need <= limit
        mid = (lo + hi) // 2
        (lo, hi) = (mid, hi) if lib.msts_solve_workspace_size(m, mid, nb, msts.MSTS_SAFE) <= limit else (lo, mid)
    n = lo
    assert lib.msts_solve_workspace_size(m, n + 64, nb, msts.MSTS_SAFE) > limit
    T, shifts, B = _rescaling_problem(m, n, 91)
    Td, sd = _dev(T), _dev(shifts)
    Xw = _dev(B)
    _, scw, sew, _ = msts.msts_solve(Td, sd, Xw, safe=True, nb=nb)
    Xs, scs, ses, st = _solve_static(f, Td, sd, B, nb)
    torch.cuda.synchronize()
    assert torch.equal(Xs, Xw) and torch.equal(ses, sew)
    del Xw
    cols = np.sort(W.rng(0, 92).choice(n, 16, replace=False))
    Xo, eo = oracle.safe_solve(T, shifts[cols], B[:, cols], nb)
    assert np.array_equal(ses.cpu().numpy()[cols], eo)
    x = Xs[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    rel = np.abs(x - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8
