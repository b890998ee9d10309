"""CPU oracle for the blocked multi-shift triangular solve (arXiv:1607.01477).

TEST INFRASTRUCTURE.  This package is the plain FP64 reference that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the library itself never
does, and it shares no code with the library.

The arithmetic lives in ``msts_oracle.c`` (plain C, binary64, no BLAS, no FMA
contraction, OpenMP across independent shifts only).  This module compiles it
with gcc on first use and exposes numpy-level wrappers.  All matrices are
complex128 in column-major (Fortran) order; only the upper triangle of U / T is
read.

Every function cites the passage of the paper it follows:
  solve              -- Eq. 2 / Alg. 1 per shift (plain definition, unblocked)
  solve_blocked      -- Alg. 3 (MultiShiftTrsm), blocked from the bottom
  safe_solve         -- Alg. 5 (SafeMultiShiftTrsm) with Alg. 4 on each block
  safe_trsv_unblocked-- Alg. 4 (SafeTrsv) on the whole shifted matrix
  trevc, trevc_columns -- Alg. 6 (TriangEig) with the strictly-upper shortcut
                        (all columns, or the listed ones bit for bit)
  back_transform     -- X = Q Z, the second half of Alg. 6 (Eig)
  gsolve             -- Alg. 8 per shift (plain definition on U - lambda_j V)
  safe_gsolve        -- Alg. 9 with the generalized Alg. 4 on each block
  gtrevc, gtrevc_columns -- Alg. 10 (GeneralizedTriangEig), triangular part
  solve_variant      -- the lower / transposed / right-hand cases (footnote
                        to Sec. 2), plain definition per shift
  safe_solve_variant -- Alg. 5 in the variant's substitution order
  pseudospectra      -- Alg. 7 (Van Loan / Lui) with Lanczos (Sec. 5)
  tridiag_max_eig    -- largest Ritz value of the Lanczos tridiagonal
  pseudospectra_1norm-- Hager/Higham 1-norm estimate of the resolvent on
                        shifted triangular solves (footnote to Sec. 5)
  portrait_grid      -- the automatic grid of SpectralPortrait (Sec. 6)
  adjoint            -- gradient of X = (U - s_j I)^{-1} b_j (not in the paper)

Parity status: every function above is pinned by ``tests/test_oracle_*.py``
and ``tests/test_golden.py`` against brute-force dense algebra, closed forms
or invariants, and ``tests/test_oracle_mutants.py`` shows that those pins fail
on planted mistakes.  No function is parity unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msts_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_c_int64 = ctypes.c_int64
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile msts_oracle.c into liboracle.so (gcc -O2, OpenMP, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_norm_inf_upper.restype = ctypes.c_double
            lib.or_delta.restype = ctypes.c_double
            lib.or_tridiag_max_eig.restype = ctypes.c_double
            lib.or_tridiag_max_eig.argtypes = [ctypes.c_int, _vp, _vp]
            lib.or_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _cz(a, name):
    if a.dtype != np.complex128:
        raise TypeError(f"{name} must be complex128")
    if not a.flags.f_contiguous:
        raise ValueError(f"{name} must be column-major (Fortran order)")
    return a


def _ld(a):
    return max(1, a.shape[0])


def _p(a):
    return a.ctypes.data_as(_vp)


def num_threads() -> int:
    return int(_load().or_num_threads())


def delta(U: np.ndarray) -> float:
    """delta = max(eps * ||U||_inf, DBL_MIN): the zero-pivot replacement (Sec. 3)."""
    U = _cz(U, "U")
    return float(_load().or_delta(_c_int64(U.shape[0]), _p(U), _c_int64(_ld(U))))


def solve(U, shifts, B, conj_trans=False):
    """x_j = (U - s_j I)^{-1} b_j by unblocked back substitution (Eq. 2, Alg. 1).

    With conj_trans, x_j = (U^H - conj(s_j) I)^{-1} b_j by forward substitution
    (the lower-triangular case of the footnote in Sec. 2).  Returns a new array.
    """
    U = _cz(U, "U")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    _load().or_multishift_solve(_c_int64(m), _p(U), _c_int64(_ld(U)), _c_int64(n), _p(s),
                                _p(X), _c_int64(_ld(X)), ctypes.c_int(1 if conj_trans else 0))
    return X


def solve_blocked(U, shifts, B, nb):
    """Alg. 3 (MultiShiftTrsm), blocked from the bottom with block size nb."""
    U = _cz(U, "U")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    _load().or_multishift_solve_blocked(_c_int64(m), _p(U), _c_int64(_ld(U)), _c_int64(n),
                                        _p(s), _p(X), _c_int64(_ld(X)), _c_int64(nb))
    return X


def safe_solve(U, shifts, B, nb, shortcut=False):
    """Alg. 5 (SafeMultiShiftTrsm): (U - s_j I) x_j = 2^-e_j b_j.

    Returns (X, e) with e the int32 scale exponents (s_j = 2^-e_j).
    shortcut declares column j of B zero in rows >= j (Alg. 6's right-hand sides).
    """
    U = _cz(U, "U")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    e = np.zeros(n, dtype=np.int32)
    _load().or_safe_multishift_solve(_c_int64(m), _p(U), _c_int64(_ld(U)), _c_int64(n), _p(s),
                                     _p(X), _c_int64(_ld(X)), _c_int64(nb),
                                     ctypes.c_int(1 if shortcut else 0), _p(e))
    return X, e


_SIDE = {"left": 0, "right": 1}
_UPLO = {"upper": 0, "lower": 1}
_TRANS = {"N": 0, "T": 1, "C": 2}


def _variant_args(A, side, uplo, trans, B):
    A = _cz(A, "A")
    if side not in _SIDE or uplo not in _UPLO or trans not in _TRANS:
        raise ValueError("side in {left,right}, uplo in {upper,lower}, trans in {N,T,C}")
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m = A.shape[0]
    n = X.shape[1] if side == "left" else X.shape[0]
    if (X.shape[0] if side == "left" else X.shape[1]) != m:
        raise ValueError("B does not match A")
    return A, X, m, n


def solve_variant(A, shifts, B, side="left", uplo="upper", trans="N"):
    """The triangular variants of the footnote to Sec. 2: M_j = op(A) - s_j I
    with op(A) in {A, A^T, A^H}, A upper or lower triangular; left side
    M_j x_j = b_j (columns of the m x n B), right side x_j^T M_j = b_j^T (rows
    of the n x m B).  Plain substitution per shift.  Returns a new array."""
    A, X, m, n = _variant_args(A, side, uplo, trans, B)
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    _load().or_solve_variant(ctypes.c_int(_SIDE[side]), ctypes.c_int(_UPLO[uplo]), ctypes.c_int(_TRANS[trans]),
                             _c_int64(m), _c_int64(n), _p(A), _c_int64(_ld(A)), _p(s), _p(X), _c_int64(_ld(X)))
    return X


def safe_solve_variant(A, shifts, B, nb, side="left", uplo="upper", trans="N"):
    """Alg. 5 for every variant, run in the variant's substitution order (the
    operator written as an upper-triangular matrix in that order).  Returns
    (X, e): M_j x_j = 2^-e_j b_j (left) or x_j^T M_j = 2^-e_j b_j^T (right)."""
    A, X, m, n = _variant_args(A, side, uplo, trans, B)
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    e = np.zeros(n, dtype=np.int32)
    _load().or_safe_solve_variant(ctypes.c_int(_SIDE[side]), ctypes.c_int(_UPLO[uplo]),
                                  ctypes.c_int(_TRANS[trans]), _c_int64(m), _c_int64(n), _p(A),
                                  _c_int64(_ld(A)), _p(s), _p(X), _c_int64(_ld(X)), _c_int64(nb), _p(e))
    return X, e


def safe_trsv_unblocked(U, shifts, B):
    """Alg. 4 (SafeTrsv) on the whole U - s_j I, column by column.  Returns (X, e)."""
    U = _cz(U, "U")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    e = np.zeros(n, dtype=np.int32)
    _load().or_safe_trsv_unblocked(_c_int64(m), _p(U), _c_int64(_ld(U)), _c_int64(n), _p(s),
                                   _p(X), _c_int64(_ld(X)), _p(e))
    return X, e


def trevc(T, nb):
    """Alg. 6 (TriangEig): upper-triangular eigenvectors Z with diag(Z) = s.

    Returns (Z, e, scales) with scales = 2^-e (0 where it underflows).
    """
    T = _cz(T, "T")
    m = T.shape[0]
    Z = np.zeros((m, m), dtype=np.complex128, order="F")
    e = np.zeros(m, dtype=np.int32)
    sc = np.zeros(m, dtype=np.float64)
    _load().or_trevc(_c_int64(m), _p(T), _c_int64(_ld(T)), _p(Z), _c_int64(_ld(Z)),
                     _c_int64(nb), _p(e), _p(sc))
    return Z, e, sc


def gsolve(U, V, shifts, B):
    """Alg. 8 per shift (plain definition): x_j = (U - s_j V)^{-1} b_j."""
    U = _cz(U, "U")
    V = _cz(V, "V")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    _load().or_gmultishift_solve(_c_int64(m), _p(U), _c_int64(_ld(U)), _p(V), _c_int64(_ld(V)), _c_int64(n),
                                 _p(s), _p(X), _c_int64(_ld(X)))
    return X


def safe_gsolve(U, V, shifts, B, nb, shortcut=False):
    """Alg. 9 (SafeGeneralizedMultiShiftTrsm): (U - s_j V) x_j = 2^-e_j b_j; returns (X, e)."""
    U = _cz(U, "U")
    V = _cz(V, "V")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    X = np.array(B, dtype=np.complex128, order="F", copy=True)
    m, n = X.shape
    e = np.zeros(n, dtype=np.int32)
    _load().or_safe_gmultishift_solve(_c_int64(m), _p(U), _c_int64(_ld(U)), _p(V), _c_int64(_ld(V)),
                                      _c_int64(n), _p(s), _p(X), _c_int64(_ld(X)), _c_int64(nb),
                                      ctypes.c_int(1 if shortcut else 0), _p(e))
    return X, e


def gtrevc(T, S, nb):
    """Alg. 10 (GeneralizedTriangEig): returns (Z, lam, e, scales) with
    lam = diag(T) ./ diag(S), T Z(:,j) = lam_j S Z(:,j), diag(Z) = 2^-e."""
    T = _cz(T, "T")
    S = _cz(S, "S")
    m = T.shape[0]
    Z = np.zeros((m, m), dtype=np.complex128, order="F")
    lam = np.zeros(m, dtype=np.complex128)
    e = np.zeros(m, dtype=np.int32)
    sc = np.zeros(m, dtype=np.float64)
    _load().or_gtrevc(_c_int64(m), _p(T), _c_int64(_ld(T)), _p(S), _c_int64(_ld(S)), _p(Z), _c_int64(_ld(Z)),
                      _p(lam), _c_int64(nb), _p(e), _p(sc))
    return Z, lam, e, sc


def gtrevc_columns(T, S, cols, nb):
    """Alg. 10 for the listed columns only: returns (Zc, lam, e) with Zc[:, c]
    the generalized eigenvector cols[c] exactly as ``gtrevc`` computes it."""
    T = _cz(T, "T")
    S = _cz(S, "S")
    m = T.shape[0]
    cc = np.ascontiguousarray(cols, dtype=np.int64)
    Zc = np.zeros((m, cc.size), dtype=np.complex128, order="F")
    lam = np.zeros(cc.size, dtype=np.complex128)
    e = np.zeros(cc.size, dtype=np.int32)
    _load().or_gtrevc_columns(_c_int64(m), _p(T), _c_int64(_ld(T)), _p(S), _c_int64(_ld(S)), _c_int64(cc.size),
                              _p(cc), _p(Zc), _c_int64(_ld(Zc)), _p(lam), _c_int64(nb), _p(e))
    return Zc, lam, e


def back_transform(Q, Z):
    """X = Q triu(Z) (the eigenvectors of A = Q T Q^H from those of T, Alg. 6)."""
    Q = _cz(Q, "Q")
    Z = _cz(Z, "Z")
    m = Q.shape[0]
    X = np.zeros((m, m), dtype=np.complex128, order="F")
    _load().or_back_transform(_c_int64(m), _p(Q), _c_int64(_ld(Q)), _p(Z), _c_int64(_ld(Z)), _p(X),
                              _c_int64(_ld(X)))
    return X


def pseudospectra(T, z, V0, iters):
    """Alg. 7 (Van Loan / Lui): sigma_min(T - z_p I) for every grid point z_p.

    V0 (m x N) holds the Lanczos start vectors (normalised inside).  Returns
    (sigma_min, alpha, beta, steps) with alpha/beta of shape (N, iters).
    """
    T = _cz(T, "T")
    V0 = _cz(V0, "V0")
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    m = T.shape[0]
    N = zz.shape[0]
    sig = np.zeros(N, dtype=np.float64)
    al = np.zeros((N, iters), dtype=np.float64)
    be = np.zeros((N, iters), dtype=np.float64)
    st = np.zeros(N, dtype=np.int32)
    _load().or_pseudospectra(_c_int64(m), _p(T), _c_int64(_ld(T)), _c_int64(N), _p(zz), _p(V0),
                             _c_int64(_ld(V0)), ctypes.c_int(iters), _p(sig), _p(al), _p(be),
                             _p(st))
    return sig, al, be, st


def pseudospectra_1norm(T, z, Q=None):
    """1-norm pseudospectra (footnote to Sec. 5): Hager/Higham estimates of
    ||Q (T - z_p I)^{-1} Q^H||_1 for every grid point (Q = I when None).
    Returns (est, kind, steps): kind = j when est = ||R e_j||_1, -1 for the
    start vector e/m, -2 for the alternative vector; steps = R^H applications."""
    T = _cz(T, "T")
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    m, N = T.shape[0], zz.shape[0]
    Qa = None if Q is None else _cz(Q, "Q")
    est = np.zeros(N, dtype=np.float64)
    kind = np.zeros(N, dtype=np.int32)
    steps = np.zeros(N, dtype=np.int32)
    _load().or_pseudospectra_1norm(_c_int64(m), _p(T), _c_int64(_ld(T)), None if Qa is None else _p(Qa),
                                   _c_int64(1 if Qa is None else _ld(Qa)), _c_int64(N), _p(zz), _p(est),
                                   _p(kind), _p(steps))
    return est, kind, steps


def portrait_grid(T, nx, ny):
    """Automatic grid of the spectral portrait: the eigenvalue bounding box
    widened by a quarter of its larger side, nx x ny points (point k + l nx).
    Returns (z, box) with box = (xmin, xmax, ymin, ymax)."""
    T = _cz(T, "T")
    z = np.zeros(nx * ny, dtype=np.complex128)
    box = np.zeros(4, dtype=np.float64)
    _load().or_portrait_grid(_c_int64(T.shape[0]), _p(T), _c_int64(_ld(T)), _c_int64(nx), _c_int64(ny),
                             _p(z), _p(box))
    return z, box


def tridiag_max_eig(a, b):
    """Largest eigenvalue of tridiag(b, a, b) by Sturm bisection."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.size == 0:
        b = np.zeros(1)
    return float(_load().or_tridiag_max_eig(ctypes.c_int(a.size), _p(a), _p(b)))


def adjoint(U, shifts, B, GX):
    """Gradients of a real loss through X = (U - s_j I)^{-1} b_j.

    GX = dL/dRe X + i dL/dIm X.  Returns (dU, dB, ds) with dU upper triangular.
    """
    U = _cz(U, "U")
    s = np.ascontiguousarray(shifts, dtype=np.complex128)
    B = np.asfortranarray(B, dtype=np.complex128)
    GX = np.asfortranarray(GX, dtype=np.complex128)
    m, n = B.shape
    dU = np.zeros((m, m), dtype=np.complex128, order="F")
    dB = np.zeros((m, n), dtype=np.complex128, order="F")
    ds = np.zeros(n, dtype=np.complex128)
    _load().or_adjoint(_c_int64(m), _p(U), _c_int64(_ld(U)), _c_int64(n), _p(s), _p(B),
                       _c_int64(_ld(B)), _p(GX), _c_int64(_ld(GX)), _p(dU), _c_int64(_ld(dU)),
                       _p(dB), _c_int64(_ld(dB)), _p(ds))
    return dU, dB, ds


def trevc_columns(T, cols, nb):
    """Alg. 6 for the listed columns only: returns (Zc, e) with Zc[:, c] the
    eigenvector cols[c] exactly as ``trevc`` computes it."""
    T = _cz(T, "T")
    m = T.shape[0]
    cc = np.ascontiguousarray(cols, dtype=np.int64)
    Zc = np.zeros((m, cc.size), dtype=np.complex128, order="F")
    e = np.zeros(cc.size, dtype=np.int32)
    _load().or_trevc_columns(_c_int64(m), _p(T), _c_int64(_ld(T)), _c_int64(cc.size), _p(cc),
                             _p(Zc), _c_int64(_ld(Zc)), _c_int64(nb), _p(e))
    return Zc, e
