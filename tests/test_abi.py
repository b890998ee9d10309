"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/msts.h declares, and rejects invalid arguments before
launching anything."""
import ctypes
import os
import re

import pytest

import paper_1607_01477_gb300 as msts
from paper_1607_01477_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return msts.load_library()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"^\s*(?:int|size_t|uint64_t)\s+(msts_\w+)\s*\(", txt, re.M))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ["msts_solve", "msts_solve_batched", "msts_trevc", "msts_pseudospectra",
              "msts_adjoint", "msts_adjoint_batched", "msts_back_transform", "msts_version"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_version(lib):
    assert lib.msts_version() >= 10000


def test_invalid_arguments_rejected_without_launch(lib):
    P = ctypes.c_void_p(16)
    # negative m
    assert lib.msts_solve(P, 1, -1, P, 1, P, 1, None, None, 32, None, 0, None, 0, None) == -3
    # ldu < m
    assert lib.msts_solve(P, 3, 4, P, 1, P, 4, None, None, 32, None, 0, None, 0, None) == -2
    # bad nb
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, None, None, 48, None, 0, None, 0, None) == -10
    # safe without scales
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, None, None, 32, P, 1 << 20, None, 1, None) == -8
    # safe | conj_trans is not offered
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, P, P, 32, P, 1 << 20, None, 3, None) == -14
    # workspace too small for the safe solve
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, P, P, 32, P, 8, None, 1, None) == -12
    # empty problems are no-ops
    assert lib.msts_solve(None, 1, 0, None, 0, None, 1, None, None, 32, None, 0, None, 0, None) == 0
    assert lib.msts_trevc(None, 1, 0, None, 1, None, None, 32, None, 0, None, 0, None) == 0
    assert lib.msts_pseudospectra(P, 4, 4, P, 2, P, 4, 0, P, None, None, None, 32, None, 0, None, 0, None) == -8
    # unknown flag bits are rejected
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, None, None, 32, P, 1 << 20, None, 64, None) == -14


def test_workspace_sizes(lib):
    assert lib.msts_solve_workspace_size(100, 10, 32, 0) == 0
    ws = lib.msts_solve_workspace_size(100, 10, 32, 1)
    assert ws > 100 * 8 * 3
    assert lib.msts_trevc_workspace_size(64, 32, 0) == lib.msts_solve_workspace_size(64, 64, 32, 1)
    assert lib.msts_trevc_workspace_size(64, 32, 8) > lib.msts_trevc_workspace_size(64, 32, 0)
    assert lib.msts_pseudospectra_workspace_size(50, 7, 20, 32, 0) >= 21 * 50 * 7 * 16


def test_back_transform_arguments_and_workspace(lib):
    P = ctypes.c_void_p(16)
    assert lib.msts_back_transform_workspace_size(64, 0) == 0
    assert lib.msts_back_transform_workspace_size(64, 8) > 8 * 2 * 64 * 64 * 2
    assert lib.msts_back_transform_workspace_size(-1, 8) == 0
    # negative m, ldq < m, ldz < m, ldx < m, unknown flags, missing / small workspace
    assert lib.msts_back_transform(P, 4, -1, P, 4, P, 4, None, 0, None, 0, None) == -3
    assert lib.msts_back_transform(P, 3, 4, P, 4, P, 4, None, 0, None, 0, None) == -2
    assert lib.msts_back_transform(P, 4, 4, P, 3, P, 4, None, 0, None, 0, None) == -5
    assert lib.msts_back_transform(P, 4, 4, P, 4, P, 3, None, 0, None, 0, None) == -7
    assert lib.msts_back_transform(P, 4, 4, P, 4, P, 4, None, 0, None, 32, None) == -11
    assert lib.msts_back_transform(P, 4, 4, P, 4, P, 4, None, 0, None, 8, None) == -8
    assert lib.msts_back_transform(P, 4, 4, P, 4, P, 4, P, 16, None, 8, None) == -9
    assert lib.msts_back_transform(None, 1, 0, None, 1, None, 1, None, 0, None, 0, None) == 0


def test_generalized_arguments_and_workspace(lib):
    P = ctypes.c_void_p(16)
    assert lib.msts_gsolve_workspace_size(64, 8, 32, 0) == 0
    assert lib.msts_gsolve_workspace_size(64, 8, 32, 1) > lib.msts_solve_workspace_size(64, 8, 32, 1)
    assert lib.msts_gtrevc_workspace_size(64, 32, 0) == lib.msts_gsolve_workspace_size(64, 64, 32, 1)
    assert lib.msts_gtrevc_workspace_size(64, 32, 8) > lib.msts_gtrevc_workspace_size(64, 32, 0)
    assert lib.msts_gtrevc_workspace_size(64, 32, 2) == 0
    assert lib.msts_gsolve_workspace_size(64, 8, 32, 9) > lib.msts_gsolve_workspace_size(64, 8, 32, 1)
    g = lib.msts_gsolve
    # negative m, ldu < m, V missing, ldv < m, bad nb, unsupported flags, missing / small workspace
    assert g(P, 4, P, 4, -1, P, 1, P, 4, None, None, 32, None, 0, None, 0, None) == -5
    assert g(P, 3, P, 4, 4, P, 1, P, 4, None, None, 32, None, 0, None, 0, None) == -2
    assert g(P, 4, None, 4, 4, P, 1, P, 4, None, None, 32, None, 0, None, 0, None) == -3
    assert g(P, 4, P, 3, 4, P, 1, P, 4, None, None, 32, None, 0, None, 0, None) == -4
    assert g(P, 4, P, 4, 4, P, 1, P, 4, None, None, 48, None, 0, None, 0, None) == -12
    assert g(P, 4, P, 4, 4, P, 1, P, 4, None, None, 32, None, 0, None, 2, None) == -16
    assert g(P, 4, P, 4, 4, P, 1, P, 4, P, P, 32, None, 0, None, 1, None) == -13
    assert g(P, 4, P, 4, 4, P, 1, P, 4, P, P, 32, P, 8, None, 1, None) == -14
    assert g(None, 1, None, 1, 0, None, 0, None, 1, None, None, 32, None, 0, None, 0, None) == 0
    t = lib.msts_gtrevc
    assert t(P, 4, None, 4, 4, P, 4, P, P, P, 32, P, 1 << 20, None, 0, None) == -3
    assert t(P, 4, P, 4, 4, P, 4, None, P, P, 32, P, 1 << 20, None, 0, None) == -8
    assert t(P, 4, P, 4, 4, P, 4, P, P, P, 32, P, 1 << 20, None, 2, None) == -15
    assert t(None, 1, None, 1, 0, None, 1, None, None, None, 32, None, 0, None, 0, None) == 0


def test_variant_arguments_and_workspace(lib):
    P = ctypes.c_void_p(16)
    ws = lib.msts_solve_variant_workspace_size
    sw = lib.msts_solve_workspace_size
    a256 = lambda x: (x + 255) // 256 * 256
    m, n = 100, 12
    for flags in (0, 1, 8, 9):
        assert ws(0, 0, 0, m, n, 32, flags) == sw(m, n, 32, flags)                         # left/upper/N
        assert ws(1, 0, 1, m, n, 32, flags) == a256(16 * m * n) + sw(m, n, 32, flags)       # right/upper/T
        assert ws(0, 1, 0, m, n, 32, flags) == a256(16 * m * m) + a256(16 * m * n) + sw(m, n, 32, flags)
        assert ws(1, 1, 2, m, n, 32, flags) == a256(16 * m * m) + a256(16 * m * n) + sw(m, n, 32, flags)
    assert ws(0, 0, 2, m, n, 32, 0) == a256(16 * n) + sw(m, n, 32, 2)                       # conjugate-transposed engine
    assert ws(0, 0, 2, m, n, 32, 1) == a256(16 * m * m) + a256(16 * m * n) + sw(m, n, 32, 1)   # safe: reversed
    assert ws(2, 0, 0, m, n, 32, 0) == 0 and ws(0, 2, 0, m, n, 32, 0) == 0 and ws(0, 0, 3, m, n, 32, 0) == 0
    assert ws(0, 0, 0, m, n, 32, 2) == 0 and ws(0, 0, 0, m, n, 48, 0) == 0
    v = lib.msts_solve_variant
    assert v(0, 0, 5, P, 4, 4, P, 2, P, 4, None, None, 32, None, 0, None, 0, None) == -15
    assert v(0, 1, 0, P, 3, 4, P, 2, P, 4, None, None, 32, None, 0, None, 0, None) == -2
    assert v(1, 1, 0, P, 4, 4, P, 6, P, 5, None, None, 32, None, 0, None, 0, None) == -7   # right: ldb >= n
    assert v(0, 1, 0, P, 4, 4, P, 2, P, 3, None, None, 32, None, 0, None, 0, None) == -7   # left: ldb >= m
    assert v(0, 1, 0, P, 4, 4, P, 2, P, 4, None, None, 32, None, 0, None, 2, None) == -14  # no conj-trans flag
    assert v(0, 1, 0, P, 4, 4, P, 2, P, 4, None, None, 32, None, 0, None, 1, None) == -8   # safe needs scales
    assert v(0, 1, 0, P, 4, 4, P, 2, P, 4, None, None, 32, None, 0, None, 0, None) == -11  # workspace missing
    assert v(1, 1, 1, None, 1, 0, None, 0, None, 1, None, None, 32, None, 0, None, 0, None) == 0


def test_pseudospectra_1norm_and_grid_arguments(lib):
    P = ctypes.c_void_p(16)
    ws = lib.msts_pseudospectra_1norm_workspace_size
    assert ws(100, 50, 32, 0, 0) > 0 and ws(100, 50, 32, 1, 0) > ws(100, 50, 32, 0, 0)
    assert ws(100, 50, 32, 1, 8) > ws(100, 50, 32, 1, 0)                 # digit planes for the Q products
    assert ws(100, 50, 32, 0, 2) == 0 and ws(100, 50, 48, 0, 0) == 0 and ws(0, 50, 32, 0, 0) == 0
    f = lib.msts_pseudospectra_1norm
    assert f(P, 3, 4, None, 1, P, 2, P, P, P, 32, None, 0, None, 0, None) == -2
    assert f(P, 4, 4, P, 3, P, 2, P, P, P, 32, None, 0, None, 0, None) == -4      # ldq < m with Q
    assert f(P, 4, 4, None, 1, P, 2, None, P, P, 32, None, 0, None, 0, None) == -7
    assert f(P, 4, 4, None, 1, P, 2, P, P, P, 48, None, 0, None, 0, None) == -8
    assert f(P, 4, 4, None, 1, P, 2, P, P, P, 32, None, 0, None, 2, None) == -11
    assert f(P, 4, 4, None, 1, P, 2, P, P, P, 32, None, 0, None, 0, None) == -9
    assert f(None, 1, 0, None, 1, None, 0, None, None, None, 32, None, 0, None, 0, None) == 0
    g = lib.msts_portrait_grid
    assert g(P, 4, 0, 3, 3, P, P, None) == -3
    assert g(P, 3, 4, 3, 3, P, P, None) == -2
    assert g(P, 4, 4, 0, 3, P, P, None) == -4
    assert g(P, 4, 4, 3, 3, None, P, None) == -5
    assert g(P, 4, 4, 3, 3, P, None, None) == -6


def test_misaligned_pointers_rejected_without_launch(lib):
    """Complex arrays must be 16-byte aligned and the workspace 256-byte
    aligned: the kernels move complex values as 16-byte vectors, so anything
    else is refused on the host with MSTS_ERR_ALIGN (after the numbered
    argument checks) instead of reaching a kernel."""
    ERR = -1002
    P, A8, W = ctypes.c_void_p(256), ctypes.c_void_p(8), ctypes.c_void_p(1 << 12)
    big = 1 << 26
    # msts_solve: U, shifts, B misaligned; workspace misaligned
    assert lib.msts_solve(A8, 4, 4, P, 1, P, 4, None, None, 32, W, big, None, 0, None) == ERR
    assert lib.msts_solve(P, 4, 4, A8, 1, P, 4, None, None, 32, W, big, None, 0, None) == ERR
    assert lib.msts_solve(P, 4, 4, P, 1, A8, 4, None, None, 32, W, big, None, 0, None) == ERR
    assert lib.msts_solve(P, 4, 4, P, 1, P, 4, None, None, 32, ctypes.c_void_p(16), big, None, 0, None) == ERR
    # a numbered argument error is still reported first
    assert lib.msts_solve(A8, 3, 4, P, 1, P, 4, None, None, 32, W, big, None, 0, None) == -2
    # msts_trevc: T misaligned
    assert lib.msts_trevc(A8, 4, 4, P, 4, P, P, 32, W, big, None, 0, None) == ERR
    # msts_gsolve: V misaligned
    assert lib.msts_gsolve(P, 4, A8, 4, 4, P, 1, P, 4, None, None, 32, W, big, None, 0, None) == ERR
    # msts_back_transform: X misaligned (no workspace needed without the tensor flag)
    assert lib.msts_back_transform(P, 4, 4, P, 4, A8, 4, None, 0, None, 0, None) == ERR
    # msts_solve_variant: B misaligned
    assert lib.msts_solve_variant(0, 1, 0, P, 4, 4, P, 1, A8, 4, None, None, 32, W, big, None, 0, None) == ERR
    # msts_pseudospectra: the grid points misaligned
    assert lib.msts_pseudospectra(P, 4, 4, A8, 1, P, 4, 2, P, None, None, None, 32, W, big, None, 0,
                                  None) == ERR
    # msts_portrait_grid: the output grid misaligned
    assert lib.msts_portrait_grid(P, 4, 4, 2, 2, A8, P, None) == ERR
    with pytest.raises(ValueError, match="aligned"):
        msts._check(ERR, "msts_solve")


def declared_prototypes():
    """name -> (return type, [parameter types]) for every prototype in include/*.h."""
    protos = {}
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        for ret, name, params in re.findall(r"\b(int|size_t|uint64_t)\s+(msts_\w+)\s*\(([^;{]*?)\)\s*;", txt, re.S):
            params = " ".join(params.split())
            types = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
            protos[name] = (ret, types)
    return protos


def _c_kind(decl):
    """Width/sign class of a C parameter declaration or return type."""
    if "*" in decl:
        return "ptr"
    base = decl.replace("const", "").split()[0]
    return {"int64_t": ("i", 8, True), "int32_t": ("i", 4, True), "uint32_t": ("i", 4, False),
            "size_t": ("i", ctypes.sizeof(ctypes.c_size_t), False), "int": ("i", 4, True),
            "uint64_t": ("i", 8, False), "double": "f64"}[base]


def _ctypes_kind(t):
    if t is ctypes.c_void_p:
        return "ptr"
    if t is ctypes.c_double:
        return "f64"
    return ("i", ctypes.sizeof(t), t(-1).value < 0)


def test_binding_signatures_match_the_header(lib):
    """Every entry point the binding declares to ctypes has the header's
    parameter count, widths and signedness, and its return type: a 64-bit
    size or leading dimension is never passed as a 32-bit int."""
    protos = declared_prototypes()
    assert set(protos) == set(declared_functions())
    for name, (ret, params) in protos.items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, f"{name}: no ctypes signature in load_library"
        assert [_ctypes_kind(t) for t in fn.argtypes] == [_c_kind(p) for p in params], name
        assert _ctypes_kind(fn.restype) == _c_kind(ret), name


def test_static_scratch_entry_rejects_invalid_arguments_without_launch(lib):
    """msts_safe_solve_static checks its arguments on the host, numbered as
    msts_solve without the workspace arguments, before anything is launched
    (no GPU is needed for any of these calls)."""
    f = lib.msts_safe_solve_static
    P, A8 = ctypes.c_void_p(256), ctypes.c_void_p(8)
    assert f(P, 1, -1, P, 1, P, 1, P, P, 32, None, None) == -3          # negative m
    assert f(P, 3, 4, P, 1, P, 4, P, P, 32, None, None) == -2           # ldu < m
    assert f(None, 4, 4, P, 1, P, 4, P, P, 32, None, None) == -1        # no U
    assert f(P, 4, 4, None, 1, P, 4, P, P, 32, None, None) == -4        # no shifts
    assert f(P, 4, 4, P, 1, None, 4, P, P, 32, None, None) == -6        # no B
    assert f(P, 4, 4, P, 1, P, 3, P, P, 32, None, None) == -7           # ldb < m
    assert f(P, 4, 4, P, 1, P, 4, None, P, 32, None, None) == -8        # no scales
    assert f(P, 4, 4, P, 1, P, 4, P, None, 32, None, None) == -9        # no scale_exp
    assert f(P, 4, 4, P, 1, P, 4, P, P, 48, None, None) == -10          # bad nb
    assert f(A8, 4, 4, P, 1, P, 4, P, P, 32, None, None) == -1002       # misaligned U
    assert f(P, 4, 4, A8, 1, P, 4, P, P, 32, None, None) == -1002       # misaligned shifts
    assert f(P, 4, 4, P, 1, A8, 4, P, P, 32, None, None) == -1002       # misaligned B
    assert f(None, 1, 0, None, 0, None, 1, None, None, 32, None, None) == 0   # empty: no-op
    assert f(P, 4, 4, None, 0, None, 4, None, None, 32, None, None) == 0      # no shifts: no-op


def test_static_scratch_entry_rejects_oversized_problem(lib):
    """A problem whose scratch exceeds the 16 MiB static array is refused with
    MSTS_ERR_STATIC_SCRATCH before any launch.  The pointers are never
    dereferenced; the size is checked first so that the call cannot reach a
    kernel even if the limit changes."""
    m = n = 20000
    assert lib.msts_solve_workspace_size(m, n, 32, msts.MSTS_SAFE) > 16 << 20
    P = ctypes.c_void_p(256)
    assert lib.msts_safe_solve_static(P, m, m, P, n, P, m, P, P, 32, None, None) == -1001
