"""Small, seeded cases of the hot kernels for profiling with ncu.

    python -m paper_1607_01477_gb300.profile_cases diag N SAFE
        single-block solves (m = n_b = 32, N shifts, SAFE 0/1): two warm-up
        solves per diagonal-step layout, then one solve each with the one-warp
        layout, the four-warp layout at 4 lanes per shift and at 1 lane.
    python -m paper_1607_01477_gb300.profile_cases trevc LAYOUT
        one safe TREVC of the 4096 workload on the tensor-core path after one
        warm-up, with the given diagonal-step layout (0, -1, 1, 2, 4).
    python -m paper_1607_01477_gb300.profile_cases pseudo N
        the pseudospectra workload's matrix (2000 x 2000) at the first N grid
        points, 2 Lanczos steps, tensor-core path, after one warm-up.
    python -m paper_1607_01477_gb300.profile_cases mixed M N
        one mixed-precision solve of workload 3's distributions at order M with
        N shifts (tensor-core low-precision product and residual), after one
        warm-up.

Every case runs through the binding (the library's C ABI) and prints "done".
"""
from __future__ import annotations

import sys

import torch

from . import colmajor, load_library, msts_pseudospectra, msts_solve, msts_solve_mixed, msts_trevc
from . import MSTS_RESIDUAL_OZAKI
from . import workloads as W


def _dev(a, dev):
    return colmajor(torch.from_numpy(a).to(dev)) if a.ndim == 2 else torch.from_numpy(a).to(dev)


def diag(n: int, safe: bool):
    lib = load_library()
    dev = torch.device("cuda", 0)
    T = W.trevc_problem(32, seed=5, cluster_frac=0.0, offdiag_scale=1.0)
    g = W.rng(0, n)
    B = W.cn(g, (32, n))
    s = W.disk(g, n, 1.5)
    Ud, sd, Bd = _dev(T, dev), _dev(s, dev), _dev(B, dev)
    X = Bd.clone()
    layouts = (-1, 4, 1)
    try:
        for lay in layouts:
            lib.msts_tune_set(1, lay)
            for _ in range(2):
                msts_solve(Ud, sd, X.copy_(Bd), safe=safe, nb=32)
        torch.cuda.synchronize()
        for lay in layouts:
            lib.msts_tune_set(1, lay)
            msts_solve(Ud, sd, X.copy_(Bd), safe=safe, nb=32)
        torch.cuda.synchronize()
    finally:
        lib.msts_tune_set(1, 0)


def trevc(layout: int):
    lib = load_library()
    dev = torch.device("cuda", 0)
    Td = _dev(W.trevc_problem(4096), dev)
    try:
        lib.msts_tune_set(1, layout)
        for _ in range(2):
            msts_trevc(Td, nb=32, tensor=True)
        torch.cuda.synchronize()
    finally:
        lib.msts_tune_set(1, 0)


def pseudo(n: int):
    dev = torch.device("cuda", 0)
    T, z, V0 = W.pseudo_problem()
    Td, zd, Vd = _dev(T, dev), _dev(z[:n].copy(), dev), _dev(V0[:, :n].copy(order="F"), dev)
    for _ in range(2):
        msts_pseudospectra(Td, zd, Vd, 2, nb=32, tensor=True)
    torch.cuda.synchronize()


def mixed(m: int, n: int):
    dev = torch.device("cuda", 0)
    U, s, B = W.mixed_problem(m, n)
    Ud, sd, Bd = _dev(U, dev), _dev(s, dev), _dev(B, dev)
    for _ in range(2):
        msts_solve_mixed(Ud, sd, Bd, tol=1e-12, nb=32, flags=MSTS_RESIDUAL_OZAKI)
    torch.cuda.synchronize()


def main(argv):
    case = argv[0]
    if case == "diag":
        diag(int(argv[1]), bool(int(argv[2])))
    elif case == "trevc":
        trevc(int(argv[1]))
    elif case == "pseudo":
        pseudo(int(argv[1]))
    elif case == "mixed":
        mixed(int(argv[1]), int(argv[2]))
    else:
        raise SystemExit(f"unknown case {case}")
    print("done")


if __name__ == "__main__":
    main(sys.argv[1:])
