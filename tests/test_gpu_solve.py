"""GPU parity: the CUDA multi-shift solve (Alg. 3), its conjugate-transposed
form and the safe variant (Alg. 4/5) against the CPU oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from conftest import backward_error
from gpu_util import EPS, cond_inf, forward_close, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,n,nb", [(256, 64, 32), (1, 1, 32), (5, 3, 16), (37, 9, 16), (100, 70, 32),
                                    (200, 33, 64), (129, 40, 64), (64, 1, 32), (700, 130, 32)])
def test_plain_solve_matches_oracle(m, n, nb, tensor):
    U, s, B = W.plain_problem(m, n, seed=1000 + m + n)
    X = to_dev(B)
    _, _, _, st = msts.msts_solve(to_dev(U), to_dev(s), X, nb=nb, tensor=tensor)
    Xg = to_np(X)
    Xo = oracle.solve(U, s, B)
    err, tol = forward_close(Xg, Xo, cond_inf(U, s), m)
    assert (err <= tol).all(), (err.max(), tol.min())
    assert backward_error(U, s, Xg, B).max() <= 8 * m * EPS
    assert int(st.item()) == 0


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,n,nb", [(256, 64, 32), (37, 9, 16), (100, 20, 64), (1, 2, 32), (500, 77, 32)])
def test_conj_trans_solve_matches_oracle(m, n, nb, tensor):
    U, s, B = W.plain_problem(m, n, seed=2000 + m)
    X = to_dev(B)
    msts.msts_solve(to_dev(U), to_dev(s), X, conj_trans=True, nb=nb, tensor=tensor)
    Xg = to_np(X)
    Xo = oracle.solve(U, s, B, conj_trans=True)
    err, tol = forward_close(Xg, Xo, cond_inf(U, s), m)
    assert (err <= tol).all()
    assert backward_error(U, s, Xg, B, conj_trans=True).max() <= 8 * m * EPS


def test_full_size_plain_config_bitwise_stable_and_accurate():
    """Workload 1 at full size (256 x 256, 64 shifts, n_b = 32): every column
    against the oracle, twice in a row (the kernels are deterministic)."""
    U, s, B = W.plain_problem()
    Ud, sd = to_dev(U), to_dev(s)
    X1, X2 = to_dev(B), to_dev(B)
    msts.msts_solve(Ud, sd, X1, nb=32)
    msts.msts_solve(Ud, sd, X2, nb=32)
    assert torch.equal(X1, X2)
    Xo = oracle.solve(U, s, B)
    err, tol = forward_close(to_np(X1), Xo, cond_inf(U, s), 256)
    assert (err <= tol).all()


@pytest.mark.parametrize("m,n,nb", [(100, 12, 16), (256, 64, 32), (130, 10, 64), (33, 5, 32)])
def test_safe_solve_equals_oracle_when_nothing_scales(m, n, nb):
    U, s, B = W.plain_problem(m, n, seed=3000 + m)
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=nb)
    Xo, eo = oracle.safe_solve(U, s, B, nb)
    assert np.array_equal(to_np(se), eo) and (eo == 0).all()
    assert (to_np(sc) == 1.0).all()
    err, tol = forward_close(to_np(X), Xo, cond_inf(U, s), m)
    assert (err <= tol).all()


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("p", [0, 1, 3])
@pytest.mark.parametrize("nb", [16, 32])
def test_safe_pow2_closed_form_bitwise(p, nb, tensor):
    """Bidiagonal powers-of-two case: every value is exact, so GPU, oracle and
    closed form agree bit for bit (x(i) 2^e = 2^(40 + (p+40)(m-1-i)))."""
    m = 32 if nb == 32 else 40
    U = np.zeros((m, m), dtype=np.complex128, order="F")
    U[np.arange(m), np.arange(m)] = 2.0 ** -40
    U[np.arange(m - 1), np.arange(1, m)] = -(2.0 ** p)
    B = np.zeros((m, 1), dtype=np.complex128, order="F")
    B[m - 1, 0] = 1.0
    s = np.zeros(1, dtype=np.complex128)
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=nb, tensor=tensor)
    Xo, eo = oracle.safe_solve(U, s, B, nb)
    e = int(to_np(se)[0])
    assert e == int(eo[0]) and e > 0
    log2x = [40 + (p + 40) * (m - 1 - i) for i in range(m)]
    expect = np.array([np.ldexp(1.0, k - e) for k in log2x])
    Xg = to_np(X)[:, 0]
    assert np.array_equal(Xg.real, expect) and np.array_equal(Xo[:, 0].real, expect)
    assert int(st.item()) & 8                       # MSTS_STATUS_SCALED


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,nb", [(256, 32), (300, 16), (257, 64)])
def test_safe_solve_with_scaling_matches_oracle(m, nb, tensor):
    """Eigenvalue-like shifts on a TREVC-style matrix: overflow scaling fires;
    scale exponents match the oracle and X agrees up to rounding."""
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, 9)
    B = W.cn(g, (m, 24))
    shifts = np.diag(T)[g.permutation(m)[:24]] + 1e-9
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(T), to_dev(shifts), X, safe=True, nb=nb, tensor=tensor)
    Xo, eo = oracle.safe_solve(T, shifts, B, nb)
    eg = to_np(se)
    assert eo.max() > 0
    assert np.array_equal(eg, eo)
    Xg = to_np(X)
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8
    sc_np = np.ldexp(1.0, -eg.astype(np.int64))
    assert backward_error(T, shifts, Xg, B, scales=sc_np).max() <= 8 * m * EPS


def test_zero_pivot_status_plain_and_delta_safe():
    U, s, B = W.plain_problem(40, 3, seed=8)
    s[1] = U[17, 17]
    X = to_dev(B)
    _, _, _, st = msts.msts_solve(to_dev(U), to_dev(s), X, nb=16)
    assert int(st.item()) & 1                        # ZERO_PIVOT
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=16)
    assert int(st.item()) & 16                       # DELTA
    Xo, eo = oracle.safe_solve(U, s, B, 16)
    assert np.array_equal(to_np(se), eo)
    Xg = to_np(X)
    assert np.isfinite(Xg).all()
    assert np.abs(Xg - Xo).max() <= 1e-8 * np.abs(Xo).max()


def test_nonfinite_input_flagged():
    U, s, B = W.plain_problem(20, 2, seed=2)
    B[3, 1] = np.nan
    X = to_dev(B)
    _, _, _, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=16)
    assert int(st.item()) & 2


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("nb", [16, 32, 64])
def test_batched_uneven_sizes_match_single_solves(tensor, nb):
    probs = W.batch_problem(batch=7, m_lo=20, m_hi=150, n=9, seed=77)
    for safe in (False, True):
        dev_probs = [(to_dev(U), to_dev(s), to_dev(B)) for U, s, B in probs]
        outs, st = msts.msts_solve_batched(dev_probs, safe=safe, nb=nb, tensor=tensor)
        for (U, s, B), (_, _, Xd), o in zip(probs, dev_probs, outs):
            if safe:
                Xo, eo = oracle.safe_solve(U, s, B, nb)
                assert np.array_equal(to_np(o[1]), eo)
            else:
                Xo = oracle.solve(U, s, B)
            err, tol = forward_close(to_np(Xd), Xo, cond_inf(U, s), U.shape[0])
            assert (err <= tol).all()


@pytest.mark.parametrize("tensor", [False, True])
def test_batched_conj_trans_matches_oracle(tensor):
    probs = W.batch_problem(batch=5, m_lo=30, m_hi=200, n=6, seed=78)
    dev_probs = [(to_dev(U), to_dev(s), to_dev(B)) for U, s, B in probs]
    msts.msts_solve_batched(dev_probs, conj_trans=True, nb=32, tensor=tensor)
    for (U, s, B), (_, _, Xd) in zip(probs, dev_probs):
        Xo = oracle.solve(U, s, B, conj_trans=True)
        err, tol = forward_close(to_np(Xd), Xo, cond_inf(U, s), U.shape[0])
        assert (err <= tol).all()


def test_batched_full_workload_both_paths_backward_stable():
    """Workload 5 (64 problems, m in 256..2048, 32 shifts): the batched solve on
    the tensor cores and the batched FP64 solve both with backward error <= 8 m
    eps on every column, and two problems against the oracle."""
    probs = W.batch_problem()
    d64 = [(to_dev(U), to_dev(s), to_dev(B)) for U, s, B in probs]
    dtc = [(U_, s_, to_dev(B)) for (U_, s_, _), (_, _, B) in zip(d64, probs)]
    msts.msts_solve_batched(d64, nb=32)
    msts.msts_solve_batched(dtc, nb=32, tensor=True)
    for (_, _, X64), (_, _, Xtc), (U, s, B) in zip(d64, dtc, probs):
        x64, xtc = to_np(X64), to_np(Xtc)
        m = U.shape[0]
        assert backward_error(U, s, xtc, B).max() <= 8 * m * EPS
        assert backward_error(U, s, x64, B).max() <= 8 * m * EPS
    for i in (0, 17):
        U, s, B = probs[i]
        Xo = oracle.solve(U, s, B)
        err, tol = forward_close(to_np(dtc[i][2]), Xo, cond_inf(U, s), U.shape[0])
        assert (err <= tol).all()


def test_graph_capture_replays_the_batched_tensor_solve():
    """The batched tensor-core solve launches only on the given stream (the
    digit planes, the diagonal steps and the batched updates): a CUDA graph
    captures it and its replay reproduces the eager result bit for bit."""
    probs = W.batch_problem(batch=6, m_lo=40, m_hi=300, n=8, seed=79)
    dp = [(to_dev(U), to_dev(s), to_dev(B)) for U, s, B in probs]
    Xs = [B.clone() for _, _, B in dp]

    def forward():
        for X, (_, _, B) in zip(Xs, dp):
            X.copy_(B)
        msts.msts_solve_batched([(U, s, X) for (U, s, _), X in zip(dp, Xs)], nb=32, tensor=True)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        forward()
        with torch.cuda.graph(g, stream=side):
            forward()
    torch.cuda.current_stream().wait_stream(side)
    eager = [X.clone() for X in Xs]
    for X in Xs:
        X.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(Xs, eager))


def test_graph_capture_replays_the_solve():
    """The C ABI launches only on the given stream: a CUDA graph captures it."""
    U, s, B = W.plain_problem(128, 16, seed=5)
    Ud, sd = to_dev(U), to_dev(s)
    Bd = to_dev(B)
    X = to_dev(B)
    status = torch.zeros(1, dtype=torch.int32, device=X.device)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        msts.msts_solve(Ud, sd, X, nb=32, status=status)   # warm-up (sets kernel attributes)
        X.copy_(Bd)
        with torch.cuda.graph(g, stream=side):
            msts.msts_solve(Ud, sd, X, nb=32, status=status)
    torch.cuda.current_stream().wait_stream(side)
    X.copy_(Bd)
    g.replay()
    torch.cuda.synchronize()
    Xo = oracle.solve(U, s, B)
    err, tol = forward_close(to_np(X), Xo, cond_inf(U, s), 128)
    assert (err <= tol).all()


@pytest.mark.parametrize("tensor", [False, True])
def test_safe_subnormal_pivot_matches_oracle(tensor):
    """A subnormal pivot (U(i,i) - s_j = 1e-310) sends its block through the
    serial safeguarded loop; scale exponents and X still match the oracle."""
    U, s, B = W.plain_problem(96, 6, seed=21)
    U[40, 40] = 1e-310
    s[2] = 0.0
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(U), to_dev(s), X, safe=True, nb=32, tensor=tensor)
    Xo, eo = oracle.safe_solve(U, s, B, 32)
    assert eo[2] > 0
    assert np.array_equal(to_np(se), eo)
    Xg = to_np(X)
    assert np.isfinite(Xg).all()
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8


@pytest.mark.parametrize("tensor", [False, True])
def test_safe_tiny_rows_with_scaling_match_oracle(tensor):
    """Right-hand sides whose upper rows are ~1e-300 become subnormal when the
    columns are rescaled: the exact slow paths of the lazy rescaling (and of the
    tensor-core update's epilogue) keep X equal to the oracle's up to rounding."""
    m = 256
    T = W.trevc_problem(m, seed=44, cluster_frac=0.1, offdiag_scale=30.0)
    g = W.rng(0, 10)
    B = W.cn(g, (m, 24))
    B[:64, :] *= 1e-300
    shifts = np.diag(T)[g.permutation(m)[:24]] + 1e-9
    X = to_dev(B)
    _, sc, se, st = msts.msts_solve(to_dev(T), to_dev(shifts), X, safe=True, nb=32, tensor=tensor)
    Xo, eo = oracle.safe_solve(T, shifts, B, 32)
    eg = to_np(se)
    assert eo.max() > 0
    assert np.array_equal(eg, eo)
    Xg = to_np(X)
    rel = np.abs(Xg - Xo).max(axis=0) / np.abs(Xo).max(axis=0)
    assert rel.max() <= 1e-8
