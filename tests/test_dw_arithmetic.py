"""The double-word FP32 arithmetic of the FP64-class residual stencil, checked on the CPU with IEEE
float32 operations in numpy: the error-free transformations it is built from are exact (TwoSum, Knuth;
TwoProduct, here by Dekker's splitting, which gives the same exact error as the FMA form), and the Dot2
accumulation with double-word operands (Ogita, Rump and Oishi 2005) reaches ~2^-48 of the sum of the
absolute terms, the accuracy class the residual selection assumes.  This pins the method; the GPU kernel
itself is compared with the FP64 oracle in test_gpu_parity.py."""
import numpy as np

f32 = np.float32


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def split(a):  # Veltkamp/Dekker: a = hi + lo with 12-bit halves
    c = f32(f32(4097.0) * a)
    hi = f32(c - f32(c - a))
    return hi, f32(a - hi)


def two_prod(a, b):
    p = f32(a * b)
    ah, al = split(a)
    bh, bl = split(b)
    e = f32(f32(f32(f32(ah * bh) - p) + f32(ah * bl)) + f32(al * bh))
    return p, f32(e + f32(al * bl))


def fma32(a, b, c):  # correctly rounded a*b + c for float32 inputs (the product is exact in float64)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def mac(h, l, uh, ul, vh, vl):
    """acc += u v as in the kernel: leading product by TwoProduct, running sum by TwoSum, the errors
    and the cross products collected in the second word."""
    p, pe = two_prod(uh, vh)
    s, e = two_sum(h, p)
    t = f32(e + pe)
    t = fma32(uh, vl, t)
    t = fma32(ul, vh, t)
    return s, f32(l + t)


def to_dw(x):
    h = f32(x)
    return h, f32(np.float64(x) - np.float64(h))


def test_two_sum_and_two_prod_are_exact():
    rng = np.random.default_rng(7)
    for _ in range(2000):
        a, b = (f32(v) for v in rng.standard_normal(2) * 10.0 ** rng.integers(-6, 6, 2))
        s, e = two_sum(a, b)
        assert np.float64(s) + np.float64(e) == np.float64(a) + np.float64(b)
        p, pe = two_prod(a, b)
        assert np.float64(p) + np.float64(pe) == np.float64(a) * np.float64(b)


def test_dot2_with_double_word_operands_reaches_48_bits():
    """500-term dot products of double-word numbers with heavy cancellation: the error is a small
    multiple of 2^-48 times the sum of the absolute terms (5.2 x 2^-48 = 1.9e-14 for these seeds, without
    the renormalisation the kernel adds after every hop pair; plain float32 is ~2^-24)."""
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(20):
        u = rng.standard_normal(500)
        v = rng.standard_normal(500)
        v[-1] = -np.dot(u[:-1], v[:-1]) / u[-1]  # the exact sum is ~0: all cancellation
        uw = [to_dw(x) for x in u]
        vw = [to_dw(x) for x in v]
        h, l = f32(0.0), f32(0.0)
        for (uh, ul), (vh, vl) in zip(uw, vw):
            h, l = mac(h, l, uh, ul, vh, vl)
        # reference: the double-word inputs exactly, in extended precision
        uu = np.array([np.longdouble(a) + np.longdouble(b) for a, b in uw])
        vv = np.array([np.longdouble(a) + np.longdouble(b) for a, b in vw])
        exact = np.sum(uu * vv)
        scale = float(np.sum(np.abs(uu * vv)))
        worst = max(worst, abs(float(np.longdouble(h) + np.longdouble(l) - exact)) / scale)
    assert worst < 8 * 2.0 ** -48
    assert worst > 0.0  # the test is sensitive: the result is not accidentally exact
