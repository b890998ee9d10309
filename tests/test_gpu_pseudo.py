"""GPU parity: pseudospectra by inverse Lanczos (Alg. 7) against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import workloads as W
from gpu_util import to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("tensor", [False, True])
@pytest.mark.parametrize("m,grid,nb", [(150, 5, 32), (16, 4, 16), (77, 3, 64), (1, 2, 32), (400, 6, 32)])
def test_pseudospectra_matches_oracle(m, grid, nb, tensor):
    T, z, V0 = W.pseudo_problem(m, grid=grid, seed=m)
    sig, al, be, st, status = msts.msts_pseudospectra(to_dev(T), to_dev(z), to_dev(V0), 20, nb=nb,
                                                      tensor=tensor)
    so, alo, beo, sto = oracle.pseudospectra(T, z, V0, 20)
    assert np.array_equal(to_np(st), sto)
    assert np.all(np.abs(to_np(sig) - so) <= 1e-10 * so)
    assert np.allclose(to_np(al), alo, rtol=1e-9, atol=1e-12 * np.abs(alo).max())


def test_pseudospectra_exact_for_small_matrix():
    """m <= iters: sigma_min equals the dense SVD value (the Krylov space is full)."""
    T, z, V0 = W.pseudo_problem(12, grid=4, seed=4)
    sig, *_ = msts.msts_pseudospectra(to_dev(T), to_dev(z), to_dev(V0), 20, nb=16)
    ref = np.array([np.linalg.svd(np.triu(T) - zz * np.eye(12), compute_uv=False).min() for zz in z])
    assert np.all(np.abs(to_np(sig) - ref) <= 1e-9 * ref)


@pytest.mark.parametrize("tensor", [False, True])
def test_pseudospectra_full_size_sampled_points(tensor):
    """Workload 4 at full size (2000 x 2000, 100 x 100 grid, 20 iterations):
    8 sampled grid points against the oracle run on the same start vectors."""
    T, z, V0 = W.pseudo_problem()
    sig, al, be, st, status = msts.msts_pseudospectra(to_dev(T), to_dev(z), to_dev(V0), 20, nb=32,
                                                      tensor=tensor)
    sg = to_np(sig)
    assert np.isfinite(sg).all() and (sg > 0).all()
    idx = np.array([0, 99, 4949, 5050, 7321, 9900, 9999, 2500])
    so, *_ = oracle.pseudospectra(T, z[idx], np.asfortranarray(V0[:, idx]), 20)
    assert np.all(np.abs(sg[idx] - so) <= 1e-10 * so)
