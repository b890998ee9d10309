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


def test_static_scratch_solve_matches_workspace_solve_twice():
    f = _entry()
    m, nb = 300, 32
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, 9)
    B = W.cn(g, (m, 24))
    shifts = np.diag(T)[g.permutation(m)[:24]] + 1e-9
    Td, sd = _dev(T), _dev(shifts)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):                      # the second call reuses the array
        Xw = _dev(B)
        _, scw, sew, _ = msts.msts_solve(Td, sd, Xw, safe=True, nb=nb)
        Xs = _dev(B)
        scs = torch.empty(24, dtype=torch.float64, device="cuda")
        ses = torch.empty(24, dtype=torch.int32, device="cuda")
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        rc = f(Td.data_ptr(), m, m, sd.data_ptr(), 24, Xs.data_ptr(), m, scs.data_ptr(),
               ses.data_ptr(), nb, status.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert torch.equal(ses, sew) and int(sew.max()) > 0     # scaling was exercised
        assert torch.equal(scs, scw)
        ref = Xw.cpu().numpy()
        rel = np.abs(Xs.cpu().numpy() - ref).max(axis=0) / np.abs(ref).max(axis=0)
        assert rel.max() <= 1e-8
        assert int(status.item()) & 8          # MSTS_STATUS_SCALED


def test_static_scratch_rejects_oversized_problem():
    f = _entry()
    fake = ctypes.c_void_p(256)                # never dereferenced: rejected before launch
    rc = f(fake, 20000, 20000, fake, 20000, fake, 20000, fake, fake, 32, None, None)
    assert rc == MSTS_ERR_STATIC_SCRATCH
