"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the solver's
arithmetic.  It serves the CUDA library's tests and benchmark and the CPU
oracle's tests alike.  Every generator is numpy ``Generator(PCG64(seed))`` with
``seed = 1607014770 + k`` for workload k unless a seed is given, and returns
complex128 arrays in column-major (Fortran) order.

``CN(0,1)`` below means N(0,1) + i N(0,1).  "Uniform in the disk of radius R"
means r = R sqrt(u1), theta = 2 pi u2.

Workloads (the paper has no public dataset for the solve; its experiments use
random triangular matrices, Sec. 7, which these stand in for):
  1 plain solve      U 256x256, strictly-upper CN/sqrt(m), diag in the unit disk,
                     64 shifts in the disk of radius 1.5 at distance >= 0.05 from
                     every diagonal entry, B CN(0,1), n_b = 32
  2 safe TREVC       T 4096x4096, diag in the unit disk with 5% of it in clusters
                     of 4 at spacing 1e-10, strictly-upper 10 * CN(0,1)
  3 mixed solve      U 8192x8192, strictly-upper CN/sqrt(m), diag in the annulus
                     0.5 <= |z| <= 1, 2048 shifts in the disk of radius 0.4
  4 pseudospectra    T 2000x2000, diag on the unit circle + 0.05 CN jitter,
                     strictly-upper CN/sqrt(m), 100x100 grid on [-1.5,1.5]^2,
                     20 Lanczos iterations, CN(0,1) start vectors
  5 batched adjoint  64 problems, m uniform in {256..2048}, built as workload 1
                     at size m with 32 shifts each
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1607014770


def rng(k: int, seed: int | None = None) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + k if seed is None else seed))


def cn(g: np.random.Generator, shape) -> np.ndarray:
    """CN(0,1) = N(0,1) + i N(0,1), column-major."""
    a = g.standard_normal(shape) + 1j * g.standard_normal(shape)
    return np.asfortranarray(a.astype(np.complex128))


def disk(g: np.random.Generator, n: int, radius: float = 1.0) -> np.ndarray:
    r = radius * np.sqrt(g.random(n))
    t = 2.0 * np.pi * g.random(n)
    return (r * np.exp(1j * t)).astype(np.complex128)


def annulus(g: np.random.Generator, n: int, rmin: float, rmax: float) -> np.ndarray:
    """Uniform in rmin <= |z| <= rmax (area measure)."""
    u = g.random(n)
    r = np.sqrt(rmin * rmin + (rmax * rmax - rmin * rmin) * u)
    t = 2.0 * np.pi * g.random(n)
    return (r * np.exp(1j * t)).astype(np.complex128)


def upper(g: np.random.Generator, m: int, diag: np.ndarray, scale: float) -> np.ndarray:
    """Upper-triangular m x m: strictly-upper scale * CN(0,1), the given diagonal,
    zero below the diagonal."""
    U = cn(g, (m, m)) * scale
    U = np.triu(U, 1)
    U[np.arange(m), np.arange(m)] = diag
    return np.asfortranarray(U)


def separated_shifts(g: np.random.Generator, n: int, radius: float, diag: np.ndarray,
                     min_dist: float) -> np.ndarray:
    """n shifts uniform in the disk of the given radius, each at distance
    >= min_dist from every diagonal entry (rejection sampling)."""
    out = np.empty(0, dtype=np.complex128)
    while out.size < n:
        cand = disk(g, max(2 * (n - out.size), 16), radius)
        d = np.abs(cand[:, None] - diag[None, :]).min(axis=1) if diag.size else np.full(cand.size, np.inf)
        out = np.concatenate([out, cand[d >= min_dist]])
    return np.ascontiguousarray(out[:n])


# --------------------------------------------------------------------------
# Workload 1: plain multi-shift solve
# --------------------------------------------------------------------------
def plain_problem(m: int = 256, n: int = 64, seed: int | None = None, k: int = 1,
                  shift_radius: float = 1.5, min_dist: float = 0.05):
    g = rng(k, seed)
    d = disk(g, m, 1.0)
    U = upper(g, m, d, 1.0 / np.sqrt(m))
    s = separated_shifts(g, n, shift_radius, d, min_dist)
    B = cn(g, (m, n))
    return U, s, B


# --------------------------------------------------------------------------
# Workload 2: safe triangular eigenvectors
# --------------------------------------------------------------------------
def trevc_problem(m: int = 4096, seed: int | None = None, k: int = 2,
                  cluster_frac: float = 0.05, cluster_size: int = 4,
                  spacing: float = 1e-10, offdiag_scale: float = 10.0):
    g = rng(k, seed)
    nclus = int(round(cluster_frac * m)) // cluster_size
    d = disk(g, m, 1.0)
    if nclus > 0:
        centres = disk(g, nclus, 1.0)
        members = (centres[:, None] + spacing * np.arange(cluster_size)[None, :]).ravel()
        d[: members.size] = members
    d = d[g.permutation(m)]
    T = upper(g, m, d, offdiag_scale)
    return T


# --------------------------------------------------------------------------
# Workload 3: mixed-precision multi-shift solve
# --------------------------------------------------------------------------
def mixed_problem(m: int = 8192, n: int = 2048, seed: int | None = None, k: int = 3):
    g = rng(k, seed)
    d = annulus(g, m, 0.5, 1.0)
    U = upper(g, m, d, 1.0 / np.sqrt(m))
    s = disk(g, n, 0.4)
    B = cn(g, (m, n))
    return U, s, B


# --------------------------------------------------------------------------
# Workload 4: pseudospectra
# --------------------------------------------------------------------------
def pseudo_problem(m: int = 2000, grid: int = 100, seed: int | None = None, k: int = 4,
                   extent: float = 1.5, jitter: float = 0.05):
    g = rng(k, seed)
    theta = 2.0 * np.pi * g.random(m)
    d = np.exp(1j * theta) + jitter * (g.standard_normal(m) + 1j * g.standard_normal(m))
    T = upper(g, m, d.astype(np.complex128), 1.0 / np.sqrt(m))
    x = np.linspace(-extent, extent, grid)
    X, Y = np.meshgrid(x, x)
    z = np.ascontiguousarray((X + 1j * Y).ravel().astype(np.complex128))
    V0 = cn(g, (m, z.size))
    return T, z, V0


# --------------------------------------------------------------------------
# Workload 5: batched differentiable solves of uneven sizes
# --------------------------------------------------------------------------
def batch_problem(batch: int = 64, m_lo: int = 256, m_hi: int = 2048, n: int = 32,
                  seed: int | None = None, k: int = 5):
    g = rng(k, seed)
    ms = g.integers(m_lo, m_hi + 1, size=batch)
    probs = []
    for mb in ms:
        mb = int(mb)
        d = disk(g, mb, 1.0)
        U = upper(g, mb, d, 1.0 / np.sqrt(mb))
        s = separated_shifts(g, n, 1.5, d, 0.05)
        B = cn(g, (mb, n))
        probs.append((U, s, B))
    return probs


# --------------------------------------------------------------------------
# Generalized eigenvectors of a triangular pencil (appendix, Alg. 10)
# --------------------------------------------------------------------------
def pencil_problem(m: int = 4096, seed: int | None = None, k: int = 6):
    """A triangular pencil (T, S): T as the TREVC workload (clustered unit-disk
    diagonal, strictly-upper 10 CN), S with diagonal 1 + 0.1 disk and
    strictly-upper 0.1 CN -- the shape of the factors QZ returns."""
    g = rng(k, seed)
    T = trevc_problem(m, seed=int(g.integers(1 << 30)))
    S = upper(g, m, 1.0 + disk(g, m, 0.1), 0.1)
    return T, S


# --------------------------------------------------------------------------
# Scaling study of the multi-shift solve (Sec. 7.1): U is the upper triangle of
# a Hermitian matrix with eigenvalues uniform in [1, 2]; shifts uniform in the
# disk of centre 1.5 and radius 0.5.
# --------------------------------------------------------------------------
def hermitian_upper(g: np.random.Generator, m: int, lo: float = 1.0, hi: float = 2.0) -> np.ndarray:
    q, r = np.linalg.qr(cn(g, (m, m)))
    q = q * (np.diagonal(r) / np.abs(np.diagonal(r)))[None, :]       # Haar-distributed unitary
    lam = lo + (hi - lo) * g.random(m)
    H = (q * lam[None, :]) @ q.conj().T
    return np.asfortranarray(np.triu(H))


def scaling_problem(m: int, n: int, seed: int | None = None, k: int = 7):
    g = rng(k, seed)
    U = hermitian_upper(g, m)
    s = 1.5 + disk(g, n, 0.5)
    B = np.asfortranarray(cn(g, (m, n)))
    return U, s, B


# --------------------------------------------------------------------------
# The Fox-Li operator (the pseudospectra test matrix of Sec. 7.3), from its
# definition: (A f)(x) = sqrt(iF/pi) int_{-1}^{1} exp(-iF (x - y)^2) f(y) dy,
# discretised by n-point Gauss-Legendre quadrature (nodes x_k, weights w_k)
# and symmetrised by the quadrature weights:
#   A_jk = sqrt(iF/pi) sqrt(w_j) exp(-iF (x_j - x_k)^2) sqrt(w_k).
# --------------------------------------------------------------------------
def fox_li(n: int = 100, F: float = 10.0) -> np.ndarray:
    x, w = np.polynomial.legendre.leggauss(n)
    sw = np.sqrt(w)
    c = np.sqrt(1j * F / np.pi)
    d = x[:, None] - x[None, :]
    return np.asfortranarray(c * (np.exp(-1j * F * d * d) * (sw[:, None] * sw[None, :])))
