"""CPU model of the closed form the diagonal-block step uses for Alg. 4's
rescaling decisions on one block (csrc/msts_diag_util.cuh, alg4_block_ka),
checked against the serial decision chain it replaces.

The chain (Alg. 4, decisions replayed after the block is solved in a scaling of
its own, exponent Kown): G = G0, Ka = 0; for each row, if the ratio exponent
em_i - Ka reaches Omega's, Ka rises to em_i - (960 - 1) and G is scaled down;
then G += a_i 2^(Kown - Ka) in FP64, and if G >= Omega, Ka rises by e(G) - 959.
The closed form claims Ka = max(0, max em_i - 959, e(S_N) - 959), S_N the
running FP64 sum of G0 and the a_i 2^Kown, with e(S_N) decided from an FP32
estimate unless S_N is within 2^-15 of a power of two.  The model follows the
kernel's arithmetic: a_i = fl(|x_i| C_i) in FP64 for the chain, and the
estimate from the leading 23 significand bits of x_i and C_i in FP32.  The
ratio exponents em_i themselves come from an FP32 estimate of |y_i| / |p_i|
(ratio_exp_est), which must equal the FP64 routine wherever it decides.
"""
import math

import numpy as np

OMEGA_EXP = 960
NONE = -(1 << 28)


def exp2_of(x: float) -> int:
    """Unbiased exponent of a positive normal double."""
    return math.frexp(x)[1] - 1


def chain(G0, a, em, kown):
    Ka, G = 0, G0
    for ai, emi in zip(a, em):
        eM = emi - Ka
        if eM >= OMEGA_EXP:
            kk = eM - (OMEGA_EXP - 1)
            Ka += kk
            G = math.ldexp(G, -kk)
        G = G + math.ldexp(ai, kown - Ka)
        if G >= math.ldexp(1.0, OMEGA_EXP):
            kk = max(1, exp2_of(G) - (OMEGA_EXP - 1))
            Ka += kk
            G = math.ldexp(G, -kk)
    return Ka


def lead_f(v: float):
    """(f, e) with |v| ~= f 2^e, f in [1, 2) from 23 leading significand bits."""
    if v == 0.0:
        return np.float32(0.0), NONE
    m, e = math.frexp(abs(v))                    # m in [0.5, 1)
    f = math.floor(m * 2.0 ** 24) / 2.0 ** 23     # 1.xxx with 23 fraction bits
    return np.float32(f), e - 1


def scale_down(f, d):
    if f == 0.0 or d < -40:
        return np.float32(0.0)
    return np.float32(math.ldexp(float(f), d))


def abs_prod_est(z: complex, c: float):
    fx, ex = lead_f(z.real)
    fy, ey = lead_f(z.imag)
    fc, ec = lead_f(c)
    E = max(ex, ey)
    if fc == 0.0 or E == NONE:
        return np.float32(0.0), NONE
    a, b = scale_down(fx, ex - E), scale_down(fy, ey - E)
    t = np.float32(np.sqrt(np.float32(np.float32(a * a) + np.float32(b * b)))) * fc
    return np.float32(t), E + ec


def closed(G0, x, c, em, kown):
    terms = []
    for z, ci in zip(x, c):
        t, e = abs_prod_est(z, ci)
        if t != 0.0:
            if e < -1020:
                return None
            terms.append((t, e + kown))
    tg, eg = lead_f(G0)
    if tg != 0.0:
        terms.append((tg, eg))
    Ka = max(0, max(em) - (OMEGA_EXP - 1))
    if not terms:
        return Ka
    tmax = max(e for _, e in terms)
    tmin = min(e for _, e in terms)
    s = np.float32(0.0)
    for t, e in terms:
        s = np.float32(s + scale_down(t, e - tmax))
    m, es = math.frexp(float(s))
    man = int((m * 2.0 - 1.0) * 2 ** 23)
    if man < 256 or man > 0x7FFFFF - 256:
        return None
    Ka = max(Ka, tmax + es - 1 - (OMEGA_EXP - 1))
    return Ka if tmin - Ka >= -1020 else None


def random_block(g, rows):
    """Values spread over a wide range around Omega, as in a rescaling block."""
    top = g.integers(880, 1000)
    kown = int(g.integers(0, 200)) if g.random() < 0.3 else 0
    x = [complex(g.standard_normal() * 2.0 ** (top - kown - g.integers(0, 60)),
                 g.standard_normal() * 2.0 ** (top - kown - g.integers(0, 60))) for _ in range(rows)]
    c = [abs(g.standard_normal()) * 2.0 ** int(g.integers(-8, 8)) for _ in range(rows)]
    a = [abs(z) * ci for z, ci in zip(x, c)]                 # fl(fl(|x|) C), FP64
    G0 = abs(g.standard_normal()) * 2.0 ** int(g.integers(top - 80, top))
    em = [int(g.integers(800, 1000)) if g.random() < 0.2 else -(1 << 28) for _ in range(rows)]
    return G0, x, c, a, em, kown


def test_closed_form_equals_the_chain_on_random_blocks():
    g = np.random.default_rng(1607)
    decided = 0
    n = 4000
    for _ in range(n):
        rows = int(g.integers(1, 33))
        G0, x, c, a, em, kown = random_block(g, rows)
        ka = closed(G0, x, c, em, kown)
        if ka is not None:
            decided += 1
            assert ka == chain(G0, a, em, kown)
    assert decided >= 0.99 * n


def test_closed_form_at_sums_just_below_and_above_omega():
    """Blocks whose full sum lands within a few percent of Omega on either side:
    the chain rescales exactly when the sum reaches it."""
    g = np.random.default_rng(7)
    hits = 0
    for _ in range(2000):
        rows = int(g.integers(2, 33))
        target = math.ldexp(1.0, OMEGA_EXP) * (1.0 + (g.random() - 0.5) * 0.1)
        w = g.random(rows)
        w /= w.sum()
        a = [float(target * wi) for wi in w]
        x = [complex(ai, 0.0) for ai in a]
        c = [1.0] * rows
        em = [-(1 << 28)] * rows
        ka = closed(0.0, x, c, em, 0)
        if ka is not None:
            assert ka == chain(0.0, a, em, 0)
            hits += ka > 0
    assert hits > 500


def test_no_term_no_rescale_and_ratio_tests_alone():
    assert closed(0.0, [0j, 0j], [1.0, 1.0], [-(1 << 28)] * 2, 0) == 0
    em = [-(1 << 28), 1000, 970]
    x = [complex(1.0, 1.0)] * 3
    a = [abs(z) for z in x]
    assert closed(1.0, x, [1.0] * 3, em, 0) == chain(1.0, a, em, 0) == 1000 - 959


def ratio_exp_fp64(y: complex, p: complex) -> int:
    """floor(log2(|y| / |p|)) from FP64 squares of the scaled components (the
    kernels' exact routine)."""
    def scaled(z):
        f = max(exp2_of(abs(z.real)) if z.real else -1022, exp2_of(abs(z.imag)) if z.imag else -1022)
        a, b = math.ldexp(z.real, -f), math.ldexp(z.imag, -f)
        n = a * a + b * b
        if n >= 4.0:
            f, n = f + 1, n * 0.25
        return f, n
    fy, ny = scaled(y)
    fp, np_ = scaled(p)
    return fy - fp - (1 if ny < np_ else 0)


def ratio_exp_fp32(y: complex, p: complex):
    """The FP32 estimate: None where it defers to the FP64 routine."""
    def est(z):
        fx, ex = lead_f(z.real)
        fy, ey = lead_f(z.imag)
        e = max(ex, ey)
        a, b = scale_down(fx, ex - e), scale_down(fy, ey - e)
        return np.float32(np.sqrt(np.float32(np.float32(a * a) + np.float32(b * b)))), e
    ty, ey = est(y)
    tp, ep = est(p)
    r = np.float32(ty / tp)
    m, er = math.frexp(float(r))
    man = int((m * 2.0 - 1.0) * 2 ** 23)
    if man < 256 or man > 0x7FFFFF - 256:
        return None
    return ey - ep + er - 1


def test_ratio_exponent_estimate_matches_fp64_routine():
    g = np.random.default_rng(99)
    decided = 0
    n = 20000
    for _ in range(n):
        y = complex(g.standard_normal(), g.standard_normal()) * 2.0 ** int(g.integers(-900, 900))
        p = complex(g.standard_normal(), g.standard_normal()) * 2.0 ** int(g.integers(-60, 4))
        if g.random() < 0.1:                      # a purely real or imaginary operand
            y = complex(y.real, 0.0)
        est = ratio_exp_fp32(y, p)
        if est is not None:
            decided += 1
            assert est == ratio_exp_fp64(y, p) == math.floor(math.log2(abs(y) / abs(p)))
    assert decided >= 0.99 * n
