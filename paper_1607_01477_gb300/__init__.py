"""GB300-native blocked multi-shift triangular solves (arXiv:1607.01477).

Thin Python binding over the C ABI of ``libmsts.so`` (``include/msts.h``).
Every function here only marshals torch tensors into the C call: all the
arithmetic runs in the library's CUDA kernels.  There is no CPU fallback; if
the library has not been built, or the tensors are not on a CUDA device, the
call raises.

Layout: complex128 matrices are column-major, i.e. a torch tensor ``A`` of
shape (m, n) with ``A.stride(0) == 1`` (``colmajor(x)`` makes such a copy).
Vectors are contiguous.  Calls are queued on the current torch CUDA stream.

Names follow the C ABI: ``msts_solve``, ``msts_solve_batched``, ``msts_trevc``,
``msts_pseudospectra``, ``msts_adjoint``, ``msts_adjoint_batched``; the
differentiable form is ``MultiShiftSolve``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

__all__ = [
    "MSTS_SAFE", "MSTS_CONJ_TRANS", "STATUS_BITS", "colmajor", "load_library", "library_path",
    "msts_solve", "msts_solve_batched", "msts_trevc", "msts_pseudospectra", "msts_adjoint",
    "msts_adjoint_batched", "msts_solve_mixed", "msts_residual", "MSTS_RESIDUAL_OZAKI",
    "MSTS_TENSOR_GEMM", "MSTS_NORMALIZE_COLUMNS", "MSTS_MIXED_FP32_GEMM", "msts_back_transform", "eig",
    "msts_gsolve", "msts_gtrevc", "geig", "msts_solve_variant",
    "msts_pseudospectra_1norm", "msts_portrait_grid", "spectral_portrait",
    "MultiShiftSolve", "multishift_solve",
    "decode_status",
]

MSTS_SAFE = 1
MSTS_CONJ_TRANS = 2
MSTS_RESIDUAL_OZAKI = 4
MSTS_TENSOR_GEMM = 8
MSTS_NORMALIZE_COLUMNS = 16
MSTS_MIXED_FP32_GEMM = 32
STATUS_BITS = {
    1: "ZERO_PIVOT", 2: "NONFINITE", 4: "RANGE", 8: "SCALED", 16: "DELTA", 32: "NOT_CONVERGED",
    64: "TIMEOUT",
}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libmsts.so")
_lib = None
_lock = threading.Lock()

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32
_u32 = ctypes.c_uint32
_sz = ctypes.c_size_t


class _Problem(ctypes.Structure):
    _fields_ = [("U", _vp), ("ldu", _i64), ("m", _i64), ("shifts", _vp), ("n", _i64),
                ("B", _vp), ("ldb", _i64), ("scales", _vp), ("scale_exp", _vp)]


class _AdjProblem(ctypes.Structure):
    _fields_ = [("U", _vp), ("ldu", _i64), ("m", _i64), ("shifts", _vp), ("n", _i64),
                ("B", _vp), ("ldb", _i64), ("GX", _vp), ("ldg", _i64), ("dU", _vp),
                ("lddu", _i64), ("dB", _vp), ("lddb", _i64), ("ds", _vp)]


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Loads libmsts.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libmsts.so is not built ({_LIB_PATH}); run __graft_entry__.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        lib.msts_version.restype = ctypes.c_int
        lib.msts_version.argtypes = []
        lib.msts_launch_count.restype = ctypes.c_uint64
        lib.msts_launch_count.argtypes = []
        lib.msts_trace_begin.restype = ctypes.c_int
        lib.msts_trace_begin.argtypes = [_i64]
        lib.msts_trace_end.restype = ctypes.c_int
        lib.msts_trace_end.argtypes = []
        lib.msts_trace_query.restype = ctypes.c_int
        lib.msts_trace_query.argtypes = [_i32, _vp, _vp, _vp, _vp]
        lib.msts_tune_set.restype = ctypes.c_int
        lib.msts_tune_set.argtypes = [_i32, _i32]
        lib.msts_inject_fallback_status.restype = ctypes.c_int
        lib.msts_inject_fallback_status.argtypes = [_u32, _vp]
        lib.msts_safe_solve_static.restype = ctypes.c_int
        lib.msts_safe_solve_static.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i32, _vp, _vp]
        lib.msts_solve_workspace_size.restype = _sz
        lib.msts_solve_workspace_size.argtypes = [_i64, _i64, _i32, _u32]
        lib.msts_solve.restype = ctypes.c_int
        lib.msts_solve.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i32, _vp, _sz,
                                   _vp, _u32, _vp]
        lib.msts_solve_batched_workspace_size.restype = _sz
        lib.msts_solve_batched_workspace_size.argtypes = [_vp, _i64, _i32, _u32]
        lib.msts_solve_batched.restype = ctypes.c_int
        lib.msts_solve_batched.argtypes = [_vp, _i64, _i32, _vp, _sz, _vp, _u32, _vp]
        lib.msts_trevc_workspace_size.restype = _sz
        lib.msts_trevc_workspace_size.argtypes = [_i64, _i32, _u32]
        lib.msts_trevc.restype = ctypes.c_int
        lib.msts_trevc.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _vp, _i32, _vp, _sz, _vp, _u32, _vp]
        lib.msts_pseudospectra_workspace_size.restype = _sz
        lib.msts_pseudospectra_workspace_size.argtypes = [_i64, _i64, _i32, _i32, _u32]
        lib.msts_pseudospectra.restype = ctypes.c_int
        lib.msts_pseudospectra.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _i32, _vp, _vp,
                                           _vp, _vp, _i32, _vp, _sz, _vp, _u32, _vp]
        lib.msts_adjoint_workspace_size.restype = _sz
        lib.msts_adjoint_workspace_size.argtypes = [_i64, _i64, _i32]
        lib.msts_adjoint.restype = ctypes.c_int
        lib.msts_adjoint.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                     _vp, _i64, _vp, _i32, _vp, _sz, _vp, _vp]
        lib.msts_adjoint_batched_workspace_size.restype = _sz
        lib.msts_adjoint_batched_workspace_size.argtypes = [_vp, _i64, _i32]
        lib.msts_adjoint_batched.restype = ctypes.c_int
        lib.msts_adjoint_batched.argtypes = [_vp, _i64, _i32, _vp, _sz, _vp, _vp]
        lib.msts_adjoint_batched_flags_workspace_size.restype = _sz
        lib.msts_adjoint_batched_flags_workspace_size.argtypes = [_vp, _i64, _i32, _u32]
        lib.msts_adjoint_batched_flags.restype = ctypes.c_int
        lib.msts_adjoint_batched_flags.argtypes = [_vp, _i64, _i32, _vp, _sz, _vp, _u32, _vp]
        lib.msts_solve_mixed_workspace_size.restype = _sz
        lib.msts_solve_mixed_workspace_size.argtypes = [_i64, _i64, _i32, _u32]
        lib.msts_solve_mixed.restype = ctypes.c_int
        lib.msts_solve_mixed.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                         ctypes.c_double, _i32, _i32, _vp, _sz, _vp, _u32, _vp,
                                         _vp, _vp, _vp]
        lib.msts_residual_workspace_size.restype = _sz
        lib.msts_residual_workspace_size.argtypes = [_i64, _i64, _u32]
        lib.msts_residual.restype = ctypes.c_int
        lib.msts_residual.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64,
                                      _vp, _sz, _vp, _u32, _vp]
        lib.msts_gsolve_workspace_size.restype = _sz
        lib.msts_gsolve_workspace_size.argtypes = [_i64, _i64, _i32, _u32]
        lib.msts_gsolve.restype = ctypes.c_int
        lib.msts_gsolve.argtypes = [_vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _i32, _vp, _sz,
                                    _vp, _u32, _vp]
        lib.msts_gtrevc_workspace_size.restype = _sz
        lib.msts_gtrevc_workspace_size.argtypes = [_i64, _i32, _u32]
        lib.msts_gtrevc.restype = ctypes.c_int
        lib.msts_gtrevc.argtypes = [_vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _i32, _vp, _sz, _vp,
                                    _u32, _vp]
        lib.msts_back_transform_workspace_size.restype = _sz
        lib.msts_back_transform_workspace_size.argtypes = [_i64, _u32]
        lib.msts_back_transform.restype = ctypes.c_int
        lib.msts_back_transform.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _sz, _vp, _u32, _vp]
        lib.msts_solve_variant_workspace_size.restype = _sz
        lib.msts_solve_variant_workspace_size.argtypes = [_i32, _i32, _i32, _i64, _i64, _i32, _u32]
        lib.msts_solve_variant.restype = ctypes.c_int
        lib.msts_solve_variant.argtypes = [_i32, _i32, _i32, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp,
                                           _i32, _vp, _sz, _vp, _u32, _vp]
        lib.msts_pseudospectra_1norm_workspace_size.restype = _sz
        lib.msts_pseudospectra_1norm_workspace_size.argtypes = [_i64, _i64, _i32, _i32, _u32]
        lib.msts_pseudospectra_1norm.restype = ctypes.c_int
        lib.msts_pseudospectra_1norm.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _vp, _vp, _i32, _vp,
                                                 _sz, _vp, _u32, _vp]
        lib.msts_portrait_grid.restype = ctypes.c_int
        lib.msts_portrait_grid.argtypes = [_vp, _i64, _i64, _i64, _i64, _vp, _vp, _vp]
        _lib = lib
        return lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def colmajor(x: torch.Tensor) -> torch.Tensor:
    """A new column-major (Fortran-order) copy of a 2-D tensor (never a view)."""
    out = torch.empty((x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()
    out.copy_(x)
    return out


def _mat(x: torch.Tensor, name: str, rows: int | None = None) -> int:
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.complex128:
        raise TypeError(f"{name} must be complex128")
    if x.dim() != 2 or (x.shape[0] > 1 and x.stride(0) != 1):
        raise ValueError(f"{name} must be a column-major 2-D tensor (stride(0) == 1)")
    if rows is not None and x.shape[0] != rows:
        raise ValueError(f"{name} must have {rows} rows")
    return max(1, x.stride(1) if x.shape[1] > 1 else x.shape[0])


def _vec(x: torch.Tensor, name: str, dtype=torch.complex128):
    if not x.is_cuda or x.dtype != dtype or x.dim() != 1 or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous 1-D CUDA {dtype} tensor")


def _ptr(x: torch.Tensor | None):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _stream(device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor | None:
    if nbytes == 0:
        return None
    return torch.empty(nbytes + 256, dtype=torch.uint8, device=device)


def _ws_ptr(ws):
    if ws is None:
        return None, 0
    base = ws.data_ptr()
    aligned = (base + 255) & ~255
    return ctypes.c_void_p(aligned), ws.numel() - (aligned - base)


def _check(rc: int, fn: str):
    if rc != 0:
        if rc == -1000:
            raise RuntimeError(f"{fn}: CUDA launch failed")
        if rc == -1002:
            raise ValueError(f"{fn}: a complex array is not 16-byte aligned or the workspace not 256-byte aligned")
        raise ValueError(f"{fn}: invalid argument {-rc}")


def decode_status(status: torch.Tensor) -> list[str]:
    v = int(status.item())
    return [name for bit, name in STATUS_BITS.items() if v & bit]


def _status(device, status):
    return torch.zeros(1, dtype=torch.int32, device=device) if status is None else status


def _tuned(kind, m, n, tensor, nb):
    """(nb, context): an explicit nb as given with the library's own layout
    choice; nb=None takes the autotuner's cached choice for this call kind and
    shape (timing the candidates on first use) and applies its layout."""
    import contextlib
    if nb is not None:
        return nb, contextlib.nullcontext()
    from . import autotune
    nb, layout = autotune.choose(kind, m, n, tensor)
    return nb, autotune.applied(layout)


# --------------------------------------------------------------------------
# entry points
# --------------------------------------------------------------------------
def msts_solve(U, shifts, B, *, safe=False, conj_trans=False, nb=32, tensor=False, status=None):
    """(U - s_j I) X(:,j) = scale_j B(:,j), in place on B (Alg. 3 / Alg. 5).

    tensor=True runs the substitution GEMM on the tensor cores (MSTS_TENSOR_GEMM).
    nb=None takes the autotuner's choice of n_b and diagonal-step layout.
    Returns (B, scales, scale_exp, status); scales/scale_exp are None unless safe.
    """
    lib = load_library()
    m, n = B.shape
    ldu = _mat(U, "U", m)
    ldb = _mat(B, "B", m)
    _vec(shifts, "shifts")
    dev = B.device
    flags = ((MSTS_SAFE if safe else 0) | (MSTS_CONJ_TRANS if conj_trans else 0)
             | (MSTS_TENSOR_GEMM if tensor else 0))
    scales = torch.empty(n, dtype=torch.float64, device=dev) if safe else None
    sexp = torch.empty(n, dtype=torch.int32, device=dev) if safe else None
    nb, tuned = _tuned("safe" if safe else ("conj" if conj_trans else "plain"), m, n, tensor, nb)
    ws = _workspace(lib.msts_solve_workspace_size(m, n, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    with tuned:
        rc = lib.msts_solve(_ptr(U), ldu, m, _ptr(shifts), n, _ptr(B), ldb, _ptr(scales), _ptr(sexp),
                            nb, wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_solve")
    return B, scales, sexp, status


_SIDES = {"left": 0, "right": 1}
_UPLOS = {"upper": 0, "lower": 1}
_OPS = {"N": 0, "T": 1, "C": 2}


def msts_solve_variant(A, shifts, B, *, side="left", uplo="upper", trans="N", safe=False, nb=32,
                       tensor=False, status=None):
    """The lower-triangular and right-hand variants (footnote to Sec. 2), in
    place on B: left (op(A) - s_j I) X(:,j) = scale_j B(:,j) with B m x n;
    right X(j,:) (op(A) - s_j I) = scale_j B(j,:) with B n x m; op(A) = A, A^T
    or A^H (trans "N", "T", "C"), A upper or lower (only that triangle read).
    Returns (B, scales, scale_exp, status); scales/scale_exp are None unless safe."""
    if side not in _SIDES or uplo not in _UPLOS or trans not in _OPS:
        raise ValueError("side in {left,right}, uplo in {upper,lower}, trans in {N,T,C}")
    lib = load_library()
    m = A.shape[0]
    lda = _mat(A, "A", m)
    if side == "left":
        n = B.shape[1]
        ldb = _mat(B, "B", m)
    else:
        n = B.shape[0]
        ldb = _mat(B, "B", n)
        if B.shape[1] != m:
            raise ValueError("B must be n x m for the right side")
    _vec(shifts, "shifts")
    dev = B.device
    flags = (MSTS_SAFE if safe else 0) | (MSTS_TENSOR_GEMM if tensor else 0)
    scales = torch.empty(n, dtype=torch.float64, device=dev) if safe else None
    sexp = torch.empty(n, dtype=torch.int32, device=dev) if safe else None
    args = (_SIDES[side], _UPLOS[uplo], _OPS[trans])
    ws = _workspace(lib.msts_solve_variant_workspace_size(*args, m, n, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_solve_variant(*args, _ptr(A), lda, m, _ptr(shifts), n, _ptr(B), ldb, _ptr(scales), _ptr(sexp),
                                nb, wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_solve_variant")
    return B, scales, sexp, status


def msts_solve_batched(problems, *, safe=False, conj_trans=False, nb=32, tensor=False, status=None):
    """Solves every (U, shifts, B) of `problems` in shared launches, in place on each B.
    tensor=True runs every problem's substitution step on the tensor cores, all
    problems of a block step in one launch; nb=None takes the autotuner's choice.

    Returns (list of (scales, scale_exp) or None, status).
    """
    lib = load_library()
    arr = (_Problem * len(problems))()
    outs, keep = [], []
    dev = None
    for i, (U, s, B) in enumerate(problems):
        m, n = B.shape
        dev = B.device
        ldu, ldb = _mat(U, "U", m), _mat(B, "B", m)
        _vec(s, "shifts")
        sc = torch.empty(n, dtype=torch.float64, device=dev) if safe else None
        se = torch.empty(n, dtype=torch.int32, device=dev) if safe else None
        outs.append((sc, se) if safe else None)
        keep += [sc, se]
        arr[i] = _Problem(U.data_ptr(), ldu, m, s.data_ptr(), n, B.data_ptr(), ldb,
                          sc.data_ptr() if safe else None, se.data_ptr() if safe else None)
    if not problems:
        return [], status
    flags = (MSTS_SAFE if safe else 0) | (MSTS_CONJ_TRANS if conj_trans else 0) | (MSTS_TENSOR_GEMM if tensor else 0)
    nb, tuned = _tuned("batched", max(B.shape[0] for _, _, B in problems), len(problems), tensor, nb)
    ws = _workspace(lib.msts_solve_batched_workspace_size(arr, len(problems), nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    with tuned:
        rc = lib.msts_solve_batched(arr, len(problems), nb, wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_solve_batched")
    return outs, status


def msts_trevc(T, *, nb=32, tensor=False, status=None):
    """Triangular eigenvectors (Alg. 6): returns (Z, scales, scale_exp, status).

    tensor=True runs the substitution GEMM on the tensor cores (MSTS_TENSOR_GEMM);
    nb=None takes the autotuner's choice of n_b and diagonal-step layout."""
    lib = load_library()
    m = T.shape[0]
    ldt = _mat(T, "T", m)
    dev = T.device
    Z = colmajor(torch.empty((m, m), dtype=torch.complex128, device=dev))
    sc = torch.empty(m, dtype=torch.float64, device=dev)
    se = torch.empty(m, dtype=torch.int32, device=dev)
    flags = MSTS_TENSOR_GEMM if tensor else 0
    nb, tuned = _tuned("trevc", m, m, tensor, nb)
    ws = _workspace(lib.msts_trevc_workspace_size(m, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    with tuned:
        rc = lib.msts_trevc(_ptr(T), ldt, m, _ptr(Z), max(1, m), _ptr(sc), _ptr(se), nb, wp, wb,
                            _ptr(status), flags, _stream(dev))
    _check(rc, "msts_trevc")
    return Z, sc, se, status


def msts_gsolve(U, V, shifts, B, *, safe=False, nb=32, tensor=False, status=None):
    """Generalized multi-shift solve (Alg. 8; Alg. 9 with safe=True): B is
    overwritten with X, (U - s_j V) X(:,j) = scale_j B(:,j).  tensor=True runs
    the substitution step on the tensor cores ([U | V] against [X; -s X]).
    Returns (B, scales, scale_exp, status); scales/scale_exp are None unless safe."""
    lib = load_library()
    m, n = B.shape
    ldu = _mat(U, "U", m)
    ldv = _mat(V, "V", m)
    ldb = _mat(B, "B", m)
    dev = B.device
    s = shifts.contiguous()
    sc = torch.empty(n, dtype=torch.float64, device=dev) if safe else None
    se = torch.empty(n, dtype=torch.int32, device=dev) if safe else None
    flags = (MSTS_SAFE if safe else 0) | (MSTS_TENSOR_GEMM if tensor else 0)
    ws = _workspace(lib.msts_gsolve_workspace_size(m, n, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_gsolve(_ptr(U), ldu, _ptr(V), ldv, m, _ptr(s), n, _ptr(B), ldb, _ptr(sc), _ptr(se), nb, wp, wb,
                         _ptr(status), flags, _stream(dev))
    _check(rc, "msts_gsolve")
    return B, sc, se, status


def msts_gtrevc(T, S, *, nb=32, tensor=False, status=None):
    """Generalized triangular eigenvectors (Alg. 10): returns (Z, lam, scales,
    scale_exp, status) with lam = diag(T) / diag(S), T Z = S Z diag(lam).
    tensor=True runs the substitution step on the tensor cores."""
    lib = load_library()
    m = T.shape[0]
    ldt = _mat(T, "T", m)
    lds = _mat(S, "S", m)
    dev = T.device
    Z = colmajor(torch.empty((m, m), dtype=torch.complex128, device=dev))
    lam = torch.empty(m, dtype=torch.complex128, device=dev)
    sc = torch.empty(m, dtype=torch.float64, device=dev)
    se = torch.empty(m, dtype=torch.int32, device=dev)
    flags = MSTS_TENSOR_GEMM if tensor else 0
    ws = _workspace(lib.msts_gtrevc_workspace_size(m, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_gtrevc(_ptr(T), ldt, _ptr(S), lds, m, _ptr(Z), max(1, m), _ptr(lam), _ptr(sc), _ptr(se), nb,
                         wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_gtrevc")
    return Z, lam, sc, se, status


def geig(A, B, *, nb=32, tensor=True, device=None):
    """Generalized eigenvalues and unit-norm eigenvectors of the pencil (A, B)
    (Alg. 10 "GeneralizedEig"): the generalized Schur (QZ) factorisation
    A = Q T P^H, B = Q S P^H comes from the host library; GeneralizedTriangEig
    (msts_gtrevc) and X = P Z (msts_back_transform) run on the GPU.
    Returns (lam, X, status) with A X(:,j) = lam[j] B X(:,j)."""
    import numpy as np
    import scipy.linalg
    A = np.asarray(A.detach().cpu().numpy() if isinstance(A, torch.Tensor) else A, dtype=np.complex128)
    B = np.asarray(B.detach().cpu().numpy() if isinstance(B, torch.Tensor) else B, dtype=np.complex128)
    T, S, _, P = scipy.linalg.qz(A, B, output="complex")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    Td = colmajor(torch.from_numpy(np.asfortranarray(T)).to(dev))
    Sd = colmajor(torch.from_numpy(np.asfortranarray(S)).to(dev))
    Pd = colmajor(torch.from_numpy(np.asfortranarray(P)).to(dev))
    Z, lam, _, _, status = msts_gtrevc(Td, Sd, nb=nb, tensor=tensor)
    X, status = msts_back_transform(Pd, Z, tensor=tensor, normalize=True, status=status)
    return lam, X, status


def msts_back_transform(Q, Z, *, tensor=False, normalize=False, status=None):
    """X = Q Z (the eigenvectors of A = Q T Q^H from those of T, Alg. 6 "Eig");
    only the upper triangle of Z is read. normalize=True scales every column of
    X to unit 2-norm. Returns (X, status)."""
    lib = load_library()
    m = Q.shape[0]
    ldq = _mat(Q, "Q", m)
    ldz = _mat(Z, "Z", m)
    dev = Q.device
    X = colmajor(torch.empty((m, m), dtype=torch.complex128, device=dev))
    flags = (MSTS_TENSOR_GEMM if tensor else 0) | (MSTS_NORMALIZE_COLUMNS if normalize else 0)
    ws = _workspace(lib.msts_back_transform_workspace_size(m, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_back_transform(_ptr(Q), ldq, m, _ptr(Z), ldz, _ptr(X), max(1, m), wp, wb, _ptr(status),
                                 flags, _stream(dev))
    _check(rc, "msts_back_transform")
    return X, status


def eig(A, *, nb=32, tensor=True, device=None):
    """Eigenvalues and unit-norm eigenvectors of a general complex matrix A
    (Alg. 6 "Eig"): the Schur factorisation A = Q T Q^H comes from the host
    library (as in the paper, which takes it from LAPACK); the triangular
    eigenvectors (msts_trevc) and the back-transformation X = Q Z
    (msts_back_transform) run on the GPU. Returns (w, X, status) with w =
    diag(T) and A X(:,j) = w[j] X(:,j)."""
    import numpy as np
    import scipy.linalg
    A = np.asarray(A.detach().cpu().numpy() if isinstance(A, torch.Tensor) else A, dtype=np.complex128)
    T, Q = scipy.linalg.schur(A, output="complex")
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    Td = colmajor(torch.from_numpy(np.asfortranarray(T)).to(dev))
    Qd = colmajor(torch.from_numpy(np.asfortranarray(Q)).to(dev))
    Z, _, _, status = msts_trevc(Td, nb=nb, tensor=tensor)
    X, status = msts_back_transform(Qd, Z, tensor=tensor, normalize=True, status=status)
    return torch.diagonal(Td).clone(), X, status


def msts_pseudospectra(T, z, V0, iters=20, *, nb=32, tensor=False, status=None, workspace=None):
    """sigma_min(T - z_p I) for every grid point (Alg. 7 with Lanczos).

    nb=None takes the autotuner's choice of n_b and diagonal-step layout.
    Returns (sigma_min, alpha, beta, steps, status); alpha/beta have shape (N, iters).
    """
    lib = load_library()
    m = T.shape[0]
    ldt = _mat(T, "T", m)
    ldv = _mat(V0, "V0", m)
    _vec(z, "z")
    N = z.shape[0]
    dev = T.device
    sig = torch.empty(N, dtype=torch.float64, device=dev)
    al = torch.empty((N, iters), dtype=torch.float64, device=dev)
    be = torch.empty((N, iters), dtype=torch.float64, device=dev)
    st = torch.empty(N, dtype=torch.int32, device=dev)
    flags = MSTS_TENSOR_GEMM if tensor else 0
    nb, tuned = _tuned("pseudo", m, N, tensor, nb)
    need = lib.msts_pseudospectra_workspace_size(m, N, iters, nb, flags)
    ws = workspace if workspace is not None and workspace.numel() >= need + 256 else _workspace(need, dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    with tuned:
        rc = lib.msts_pseudospectra(_ptr(T), ldt, m, _ptr(z), N, _ptr(V0), ldv, iters, _ptr(sig),
                                    _ptr(al), _ptr(be), _ptr(st), nb, wp, wb, _ptr(status), flags,
                                    _stream(dev))
    _check(rc, "msts_pseudospectra")
    return sig, al, be, st, status


def msts_pseudospectra_1norm(T, z, Q=None, *, nb=32, tensor=True, status=None):
    """1-norm pseudospectra (footnote to Sec. 5): Hager/Higham lower-bound
    estimates of ||(z_p I - A)^{-1}||_1, A = Q T Q^H (A = T without Q).

    Returns (est, kind, steps, status): kind[p] = j when est = ||R e_j||_1,
    -1 for the start vector, -2 for the alternative vector."""
    lib = load_library()
    m = T.shape[0]
    ldt = _mat(T, "T", m)
    ldq = _mat(Q, "Q", m) if Q is not None else 1
    _vec(z, "z")
    N = z.shape[0]
    dev = T.device
    est = torch.empty(N, dtype=torch.float64, device=dev)
    kind = torch.empty(N, dtype=torch.int32, device=dev)
    steps = torch.empty(N, dtype=torch.int32, device=dev)
    flags = MSTS_TENSOR_GEMM if tensor else 0
    ws = _workspace(lib.msts_pseudospectra_1norm_workspace_size(m, N, nb, 0 if Q is None else 1, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_pseudospectra_1norm(_ptr(T), ldt, m, _ptr(Q), ldq, _ptr(z), N, _ptr(est), _ptr(kind),
                                      _ptr(steps), nb, wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_pseudospectra_1norm")
    return est, kind, steps, status


def msts_portrait_grid(T, nx, ny):
    """The automatic grid of a spectral portrait: (z, box), z of nx*ny points
    (point k + l nx), box = (xmin, xmax, ymin, ymax) on the device."""
    lib = load_library()
    m = T.shape[0]
    ldt = _mat(T, "T", m)
    dev = T.device
    z = torch.empty(nx * ny, dtype=torch.complex128, device=dev)
    box = torch.empty(4, dtype=torch.float64, device=dev)
    rc = lib.msts_portrait_grid(_ptr(T), ldt, m, nx, ny, _ptr(z), _ptr(box), _stream(dev))
    _check(rc, "msts_portrait_grid")
    return z, box


def spectral_portrait(T, nx=100, ny=100, *, norm=2, Q=None, iters=20, nb=32, tensor=True, seed=0):
    """SpectralPortrait (Sec. 6): resolvent norms of A = Q T Q^H over the
    automatic grid.  norm=2: 1/sigma_min(T - zI) by inverse Lanczos (Q does
    not change the 2-norm; iters <= 64; start vectors CN(0,1) from `seed`); norm=1: the
    Hager/Higham estimate of ||(zI - A)^{-1}||_1.  Returns (resolvent norms
    as an ny x nx array, box, status)."""
    z, box = msts_portrait_grid(T, nx, ny)
    m = T.shape[0]
    if norm == 2:
        g = torch.Generator(device=T.device).manual_seed(seed)
        V0 = colmajor(torch.randn((m, nx * ny), dtype=torch.complex128, device=T.device, generator=g))
        sig, _, _, _, status = msts_pseudospectra(T, z, V0, iters, nb=nb, tensor=tensor)
        res = 1.0 / sig
    elif norm == 1:
        res, _, _, status = msts_pseudospectra_1norm(T, z, Q, nb=nb, tensor=tensor)
    else:
        raise ValueError("norm must be 1 or 2")
    return res.reshape(ny, nx), box, status


def msts_adjoint(U, shifts, B, GX, *, nb=32, status=None):
    """Gradients of a real loss through X = (U - s_j I)^{-1} B(:,j): (dU, dB, ds, status)."""
    lib = load_library()
    m, n = B.shape
    ldu, ldb, ldg = _mat(U, "U", m), _mat(B, "B", m), _mat(GX, "GX", m)
    _vec(shifts, "shifts")
    dev = B.device
    dU = colmajor(torch.empty((m, m), dtype=torch.complex128, device=dev))
    dB = colmajor(torch.empty((m, n), dtype=torch.complex128, device=dev))
    ds = torch.empty(n, dtype=torch.complex128, device=dev)
    ws = _workspace(lib.msts_adjoint_workspace_size(m, n, nb), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_adjoint(_ptr(U), ldu, m, _ptr(shifts), n, _ptr(B), ldb, _ptr(GX), ldg, _ptr(dU),
                          max(1, m), _ptr(dB), max(1, m), _ptr(ds), nb, wp, wb, _ptr(status),
                          _stream(dev))
    _check(rc, "msts_adjoint")
    return dU, dB, ds, status


def msts_adjoint_batched(problems, *, nb=32, tensor=False, status=None):
    """problems: list of (U, shifts, B, GX).  Returns (list of (dU, dB, ds), status).
    tensor=True runs the substitution steps of both internal solves and the product
    dU = -triu(Lambda X^H) on the tensor cores."""
    lib = load_library()
    arr = (_AdjProblem * len(problems))()
    outs = []
    dev = None
    for i, (U, s, B, G) in enumerate(problems):
        m, n = B.shape
        dev = B.device
        ldu, ldb, ldg = _mat(U, "U", m), _mat(B, "B", m), _mat(G, "GX", m)
        _vec(s, "shifts")
        dU = colmajor(torch.empty((m, m), dtype=torch.complex128, device=dev))
        dB = colmajor(torch.empty((m, n), dtype=torch.complex128, device=dev))
        ds = torch.empty(n, dtype=torch.complex128, device=dev)
        outs.append((dU, dB, ds))
        arr[i] = _AdjProblem(U.data_ptr(), ldu, m, s.data_ptr(), n, B.data_ptr(), ldb, G.data_ptr(),
                             ldg, dU.data_ptr(), max(1, m), dB.data_ptr(), max(1, m), ds.data_ptr())
    if not problems:
        return [], status
    flags = MSTS_TENSOR_GEMM if tensor else 0
    ws = _workspace(lib.msts_adjoint_batched_flags_workspace_size(arr, len(problems), nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_adjoint_batched_flags(arr, len(problems), nb, wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_adjoint_batched_flags")
    return outs, status


def msts_residual(U, shifts, B, X, *, ozaki=False, status=None):
    """R = B - (triu(U) - diag(s)) X; ozaki=True uses the tensor-core product."""
    lib = load_library()
    m, n = B.shape
    ldu, ldb, ldx = _mat(U, "U", m), _mat(B, "B", m), _mat(X, "X", m)
    _vec(shifts, "shifts")
    dev = B.device
    flags = MSTS_RESIDUAL_OZAKI if ozaki else 0
    R = colmajor(torch.empty((m, n), dtype=torch.complex128, device=dev))
    ws = _workspace(lib.msts_residual_workspace_size(m, n, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    rc = lib.msts_residual(_ptr(U), ldu, m, _ptr(shifts), n, _ptr(B), ldb, _ptr(X), ldx, _ptr(R),
                           max(1, m), wp, wb, _ptr(status), flags, _stream(dev))
    _check(rc, "msts_residual")
    return R, status


def msts_solve_mixed(U, shifts, B, *, tol=1e-12, max_iter=10, nb=32, flags=0, status=None):
    """Mixed-precision solve with FP64 iterative refinement (synchronous).

    flags: MSTS_RESIDUAL_OZAKI (tensor-core FP64-accurate residual) and
    MSTS_MIXED_FP32_GEMM (FP32 FMA low-precision product instead of the tensor
    cores' 3-plane split-BF16 one).

    Returns (X, info, status) with info = {"iters", "eta", "eta_before"}.
    """
    lib = load_library()
    m, n = B.shape
    ldu, ldb = _mat(U, "U", m), _mat(B, "B", m)
    _vec(shifts, "shifts")
    dev = B.device
    X = colmajor(torch.empty((m, n), dtype=torch.complex128, device=dev))
    ws = _workspace(lib.msts_solve_mixed_workspace_size(m, n, nb, flags), dev)
    wp, wb = _ws_ptr(ws)
    status = _status(dev, status)
    it = ctypes.c_int32()
    eta = ctypes.c_double()
    eta0 = ctypes.c_double()
    rc = lib.msts_solve_mixed(_ptr(U), ldu, m, _ptr(shifts), n, _ptr(B), ldb, _ptr(X), max(1, m),
                              tol, max_iter, nb, wp, wb, _ptr(status), flags, ctypes.byref(it),
                              ctypes.byref(eta), ctypes.byref(eta0), _stream(dev))
    _check(rc, "msts_solve_mixed")
    return X, {"iters": it.value, "eta": eta.value, "eta_before": eta0.value}, status


class MultiShiftSolve(torch.autograd.Function):
    """X = MultiShiftSolve.apply(U, shifts, B): X(:,j) = (triu(U) - s_j I)^{-1} B(:,j).

    Backward runs the library's adjoint (a conjugate-transposed multi-shift
    solve plus a triangular-output GEMM); X is not saved, it is recomputed.
    """

    @staticmethod
    def forward(ctx, U, shifts, B, nb=32):
        X = colmajor(B.detach())
        msts_solve(U.detach(), shifts.detach(), X, nb=nb)
        ctx.save_for_backward(U, shifts, B)
        ctx.nb = nb
        return X

    @staticmethod
    def backward(ctx, gX):
        U, shifts, B = ctx.saved_tensors
        dU, dB, ds, _ = msts_adjoint(U.detach(), shifts.detach(), B.detach(), colmajor(gX),
                                     nb=ctx.nb)
        return dU, ds, dB, None


def multishift_solve(U, shifts, B, nb=32):
    return MultiShiftSolve.apply(U, shifts, B, nb)
