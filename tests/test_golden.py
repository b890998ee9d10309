"""The oracle against the closed-form fixtures in tests/golden/closed_forms.json."""
import json
import os

import numpy as np

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "closed_forms.json")))


def test_bidiagonal_pow2_fixture():
    for c in G["bidiagonal_pow2"]["cases"]:
        m, d, p, nb = c["m"], c["d"], c["p"], c["nb"]
        U = np.zeros((m, m), dtype=np.complex128, order="F")
        U[np.arange(m), np.arange(m)] = 2.0 ** d
        U[np.arange(m - 1), np.arange(1, m)] = -(2.0 ** p)
        b = np.zeros((m, 1), dtype=np.complex128, order="F")
        b[-1, 0] = 1.0
        s = np.zeros(1, dtype=np.complex128)
        X, e = oracle.safe_trsv_unblocked(U, s, b) if nb == 0 else oracle.safe_solve(U, s, b, nb)
        expect = [np.ldexp(1.0, -d + (p - d) * (m - 1 - i) - int(e[0])) for i in range(m)]
        assert np.array_equal(X[:, 0].real, np.array(expect))


def test_trevc_2x2_fixture():
    for c in G["trevc_2x2"]["cases"]:
        a, b, cc = (complex(*c[k]) for k in ("a", "b", "c"))
        T = np.asfortranarray(np.array([[a, b], [0, cc]], dtype=np.complex128))
        Z, e, sc = oracle.trevc(T, 32)
        assert Z[0, 0] == 1 and Z[1, 0] == 0 and Z[1, 1] == 1
        assert abs(Z[0, 1] - b / (cc - a)) <= 4e-16 * abs(b / (cc - a))


def test_diagonal_pseudospectra_fixture():
    for c in G["diagonal_pseudospectra"]["cases"]:
        d = np.array([complex(*x) for x in c["diag"]])
        z = np.array([complex(*x) for x in c["z"]])
        T = np.asfortranarray(np.diag(d))
        V0 = np.asfortranarray(np.ones((d.size, z.size), dtype=np.complex128) + 0.1j)
        sig, *_ = oracle.pseudospectra(T, z, V0, 20)
        assert np.allclose(sig, c["sigma_min"], rtol=1e-12, atol=0)


def test_safe_rescale_exponent_fixture():
    """The rescale exponent of Alg. 4 / Alg. 5 itself, not only x up to scale:
    e = 2 exactly (the smallest k with 2^-k G < Omega), x exact."""
    f = G["safe_rescale_exponent_2x2"]
    U = np.asfortranarray(np.array([[complex(*z) for z in row] for row in f["U"]], dtype=np.complex128))
    b = np.zeros((2, 1), dtype=np.complex128, order="F")
    b[f["b_log2"]["row"], 0] = np.ldexp(f["b_log2"]["mantissa"], f["b_log2"]["exp2"])
    s = np.zeros(1, dtype=np.complex128)
    x_expect = np.array([np.ldexp(v["mantissa"], v["exp2"]) for v in f["expect"]["x"]])
    for c in f["cases"]:
        X, e = oracle.safe_trsv_unblocked(U, s, b) if c["nb"] == 0 else oracle.safe_solve(U, s, b, c["nb"])
        assert int(e[0]) == f["expect"]["e"], c
        assert np.array_equal(X[:, 0], x_expect.astype(np.complex128)), c
        assert np.array_equal(np.triu(U) @ X[:, 0], np.ldexp(1.0, -int(e[0])) * b[:, 0])


def test_safe_gsolve_rescale_exponent_fixture():
    """The same exact exponent for the safe generalized solve (Alg. 9), with the
    off-diagonal growth coming from V only, so the |lambda| ||V|| part of the
    bounds decides the rescale."""
    f = G["safe_gsolve_rescale_exponent_2x2"]
    mat = lambda key: np.asfortranarray(np.array([[complex(*z) for z in row] for row in f[key]], dtype=np.complex128))
    U, V = mat("U"), mat("V")
    lam = np.array([complex(*f["lambda"])])
    b = np.zeros((2, 1), dtype=np.complex128, order="F")
    b[f["b_log2"]["row"], 0] = np.ldexp(f["b_log2"]["mantissa"], f["b_log2"]["exp2"])
    x_expect = np.array([np.ldexp(v["mantissa"], v["exp2"]) for v in f["expect"]["x"]], dtype=np.complex128)
    for c in f["cases"]:
        X, e = oracle.safe_gsolve(U, V, lam, b, c["nb"])
        assert int(e[0]) == f["expect"]["e"], c
        assert np.array_equal(X[:, 0], x_expect), c
