"""Host emulation of the double-word building blocks used by the GPU kernels
(no GPU): the integer split of an FP64 value into two floats (the layout
conversion of double-word plan runs and of the complex128 expectation passes)
and the FMA-based product and sum, checked against exact rational arithmetic
at the stated error bounds."""
from fractions import Fraction

import numpy as np

F = np.float32


def split_bits(x):
    """numpy mirror of the device split: h = the top 24 significant bits of x
    (truncated), l = the next 29 bits rounded to 23, |x - h - l| <= 2^-47 |x|."""
    b = np.float64(x).view(np.uint64)
    hi32, lo32 = np.uint32(b >> np.uint64(32)), np.uint32(b & np.uint64(0xFFFFFFFF))
    e = (int(hi32) >> 20) & 0x7FF
    if e < 920:
        return F(0), F(0)
    sh = (int(hi32) - (896 << 20)) & 0xFFFFFFFF
    fun = ((sh << 3) | (int(lo32) >> 29)) & 0xFFFFFFFF
    hb = (int(hi32) & 0x80000000) | (fun & 0x7FFFFFFF)
    mb = ((hb & 0xFF800000) - (23 << 23)) & 0xFFFFFFFF
    q = ((int(lo32) & 0x1FFFFFFF) + 32) >> 6
    a = np.uint32((mb + q) & 0xFFFFFFFF).view(np.float32)
    m = np.uint32(mb).view(np.float32)
    return np.uint32(hb).view(np.float32), F(a - m)


def two_prod_fma(a, b):
    """(ph, pl) with ph + pl = a b exactly (the FMA's exact residual)."""
    ph = F(a * b)
    pl = F(Fraction(float(a)) * Fraction(float(b)) - Fraction(float(ph)))  # what fmaf(a, b, -ph) returns
    return ph, pl


def test_split_error_bound_over_the_exponent_range():
    rng = np.random.default_rng(5)
    for _ in range(4000):
        x = float(rng.standard_normal() * 2.0 ** rng.integers(-100, 100))
        if abs(x) < 2.0 ** -103:  # the flushed range, checked below
            continue
        h, l = split_bits(x)
        err = abs(Fraction(x) - Fraction(float(h)) - Fraction(float(l)))
        assert err <= Fraction(abs(x)) * Fraction(1, 2 ** 47), x
        assert abs(float(l)) <= abs(float(h)) * 2.0 ** -23  # l below one unit of h's last place
    for x in (0.0, -0.0, 1.0, -1.0, 0.5, 3.0, 2.0 ** -103, 2.0 ** 60):  # exact values stay exact
        h, l = split_bits(x)
        assert float(h) + float(l) == x
    assert split_bits(2.0 ** -104) == (0.0, 0.0)  # below the range: flushed (absolute error < 2^-103)


def test_double_word_multiply_add_error():
    # fma(a, b, c) of the generated kernels: exact product of the high parts,
    # cross terms, TwoSum of the high parts, low parts in float; no final
    # renormalisation.  Error a few 2^-48 of |a b| + |c|.
    rng = np.random.default_rng(6)
    worst = 0.0
    for _ in range(3000):
        xa, xb, xc = (float(v) for v in rng.standard_normal(3))
        xc *= float(rng.choice([1.0, 1e-3, 1e3]))
        a, b, c = split_bits(xa), split_bits(xb), split_bits(xc)
        ph, pl = two_prod_fma(a[0], b[0])
        pl = F(Fraction(float(a[0])) * Fraction(float(b[1])) + Fraction(float(pl)))  # fmaf rounds once
        pl = F(Fraction(float(a[1])) * Fraction(float(b[0])) + Fraction(float(pl)))
        s = F(ph + c[0])
        v = F(s - ph)
        e = F(F(ph - F(s - v)) + F(c[0] - v))
        r = (s, F(e + F(pl + c[1])))
        exact = sum(Fraction(float(t)) for t in a) * sum(Fraction(float(t)) for t in b) + sum(
            Fraction(float(t)) for t in c)
        err = abs(Fraction(float(r[0])) + Fraction(float(r[1])) - exact)
        scale = abs(xa * xb) + abs(xc)
        worst = max(worst, float(err) / scale)
    assert worst <= 8 * 2.0 ** -48, worst
