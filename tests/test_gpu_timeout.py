"""Failure detection in the tensor-core kernels, injected from the host.

Every mbarrier wait in the tensor-core kernels is bounded. It gives up after
about two seconds, or as soon as the caller's status word holds
MSTS_STATUS_TIMEOUT, which is how a CTA that gave up tells the others. A CTA
that gives up then waits, with a time limit, for the copies and MMAs it issued,
frees its TMEM and returns; the host reads MSTS_STATUS_TIMEOUT.

These tests start a call with that bit already set in the status word (nothing
on the GPU clears it), so the kernels take the give-up path with no real fault:
the status must still carry the bit afterwards, and the next call in the same
context, with a clean status word, must be correct.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

TIMEOUT = 64   # MSTS_STATUS_TIMEOUT


def preset_status():
    return torch.full((1,), TIMEOUT, dtype=torch.int32, device="cuda")


def test_chunked_kernel_gives_up_and_the_context_stays_usable():
    """k_oz_gemm (the tensor-core residual)."""
    m, n = 320, 96
    U, s, B = W.mixed_problem(m, n, seed=5)
    X = np.asfortranarray(W.cn(W.rng(0, 6), (m, n)))
    Ud, sd, Bd, Xd = to_dev(U), to_dev(s), to_dev(B), to_dev(X)
    _, st = msts.msts_residual(Ud, sd, Bd, Xd, ozaki=True, status=preset_status())
    torch.cuda.synchronize()
    assert int(st.item()) & TIMEOUT
    R64, st64 = msts.msts_residual(Ud, sd, Bd, Xd)
    Roz, st2 = msts.msts_residual(Ud, sd, Bd, Xd, ozaki=True)
    assert int(st2.item()) == 0 and int(st64.item()) == 0
    d = np.abs(to_np(Roz) - to_np(R64))
    assert d.max() <= 1e-12 * np.abs(to_np(R64)).max()


def test_persistent_update_kernel_gives_up_and_the_context_stays_usable():
    """k_oz_update (the persistent tensor-core substitution step, n_b = 32)."""
    U, s, B = W.plain_problem(200, 40, seed=9)
    Ud, sd = to_dev(U), to_dev(s)
    Xa = to_dev(B)
    _, _, _, st = msts.msts_solve(Ud, sd, Xa, nb=32, tensor=True, status=preset_status())
    torch.cuda.synchronize()
    assert int(st.item()) & TIMEOUT
    Xt, Xf = to_dev(B), to_dev(B)
    _, _, _, st_t = msts.msts_solve(Ud, sd, Xt, nb=32, tensor=True)
    _, _, _, st_f = msts.msts_solve(Ud, sd, Xf, nb=32, tensor=False)
    assert int(st_t.item()) == 0 and int(st_f.item()) == 0
    xt, xf = to_np(Xt), to_np(Xf)
    assert np.abs(xt - xf).max() <= 1e-10 * np.abs(xf).max()


def test_call_without_status_word_is_not_cut_short_by_an_earlier_give_up():
    """A call made with status == NULL publishes its timeouts in a word of the
    library's own.  With MSTS_STATUS_TIMEOUT injected into that word from the
    host (as a give-up of an earlier call would leave it), the next tensor-core
    solve without a status word must still run to the end: its result equals
    the same solve made with a clean status word of the caller's, bit for bit."""
    lib = msts.load_library()
    U, s, B = W.plain_problem(200, 40, seed=9)
    Ud, sd = to_dev(U), to_dev(s)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    m, n = B.shape
    flags = msts.MSTS_TENSOR_GEMM
    nbytes = lib.msts_solve_workspace_size(m, n, 32, flags)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    wp = (ws.data_ptr() + 255) & ~255
    for _ in range(2):
        assert lib.msts_inject_fallback_status(TIMEOUT, stream) == 0
        Xn = to_dev(B)
        rc = lib.msts_solve(Ud.data_ptr(), m, m, sd.data_ptr(), n, Xn.data_ptr(), m, None, None, 32,
                            ctypes.c_void_p(wp), nbytes, None, flags, stream)
        assert rc == 0
        Xs = to_dev(B)
        _, _, _, st = msts.msts_solve(Ud, sd, Xs, nb=32, tensor=True)
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(Xn, Xs)
