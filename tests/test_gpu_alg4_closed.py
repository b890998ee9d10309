"""GPU: Alg. 4's rescaling decisions per diagonal block from the closed form
(the default) against the serial decision chain (MSTS_TUNE_ALG4_CHAIN = 1),
bit for bit, on every diagonal-step layout and both substitution paths, on
problems that rescale in most blocks; and on the full TREVC workload (4096,
clustered eigenvalues), where scale exponents run into the thousands."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu

MSTS_TUNE_DIAG_LANES, MSTS_TUNE_ALG4_CHAIN = 1, 2


def run(fn, layout, chain):
    lib = msts.load_library()
    assert lib.msts_tune_set(MSTS_TUNE_DIAG_LANES, layout) == 0
    assert lib.msts_tune_set(MSTS_TUNE_ALG4_CHAIN, chain) == 0
    try:
        out = fn()
        torch.cuda.synchronize()
        return out
    finally:
        assert lib.msts_tune_set(MSTS_TUNE_ALG4_CHAIN, 0) == 0
        assert lib.msts_tune_set(MSTS_TUNE_DIAG_LANES, 0) == 0


def test_knob_rejects_invalid_values():
    lib = msts.load_library()
    assert lib.msts_tune_set(MSTS_TUNE_ALG4_CHAIN, 3) == -2
    assert lib.msts_tune_set(99, 0) == -1


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("layout", [-1, 1, 2, 4])
@pytest.mark.parametrize("m,n,seed", [(300, 64, 11), (97, 40, 12), (512, 600, 13)])
def test_safe_solve_closed_form_equals_chain(layout, tensor, m, n, seed):
    scale = 30.0 if m >= 200 else 1000.0            # large enough for the order that columns rescale
    T = W.trevc_problem(m, seed=seed, cluster_frac=0.1, offdiag_scale=scale)
    g = W.rng(0, seed + 1)
    B = W.cn(g, (m, n))
    shifts = np.diag(T)[g.integers(0, m, n)] + 1e-9
    Td, sd = to_dev(T), to_dev(shifts)
    res = []
    for chain in (1, 0):
        X = to_dev(B)
        _, sc, se, st = run(lambda: msts.msts_solve(Td, sd, X, safe=True, nb=32, tensor=tensor), layout, chain)
        res.append((X, sc, se, int(st.item())))
    (X1, sc1, se1, st1), (X0, sc0, se0, st0) = res
    assert torch.equal(X0, X1) and torch.equal(sc0, sc1) and torch.equal(se0, se1) and st0 == st1
    assert int(se0.max().item()) > 0
    Xo, eo = oracle.safe_solve(T, shifts, B, 32)
    assert np.array_equal(to_np(se0), eo)


@pytest.mark.parametrize("layout", [0, -1])
def test_trevc_4096_closed_form_equals_chain(layout):
    T = W.trevc_problem(4096)
    Td = to_dev(T)
    Zc, scc, sec, _ = run(lambda: msts.msts_trevc(Td, nb=32, tensor=True), layout, 1)
    Zf, scf, sef, _ = run(lambda: msts.msts_trevc(Td, nb=32, tensor=True), layout, 0)
    assert torch.equal(Zc, Zf) and torch.equal(sec, sef) and torch.equal(scc, scf)
    assert int(sef.max().item()) > 1000
