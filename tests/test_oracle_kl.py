"""Pins of the oracle's Kenney-Laub rationals against the paper's own numbers.

Tab. 5 / Tab. 6 coefficients, the binomial / tanh forms (Eq. def_gell),
Tab. 1 / Tab. 2 polynomials, the continued fractions of Sec. 3.3, the nesting
property (Eq. nesting), the cascade coefficients of Sec. 8 and Tab. 4.
"""
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest

from oracle import kl

XS = np.concatenate([-np.logspace(-3, 2.5, 41), np.logspace(-3, 2.5, 41), [0.3, 1.0, -1.0]])


def _read(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_tab5_tab6_partial_fractions(golden_dir):
    rows = _read(golden_dir, "kl_partial_fractions_tab5_tab6.txt")
    by = {}
    for kind, n, const, w, s in rows:
        by.setdefault((int(kind), int(n)), []).append((float(Fraction(const)), float(w), float(s)))
    assert len(by) == 10
    for (kind, n), entries in by.items():
        c0, w, sig = kl.kl_coeffs(n, kind)
        assert len(w) == len(entries) == n
        for i, (cp, wp, sp) in enumerate(entries):
            assert c0 == pytest.approx(cp, rel=1e-15, abs=1e-16)
            assert w[i] == pytest.approx(wp, rel=3e-15)
            assert sig[i] == pytest.approx(sp, rel=3e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 8, 12, 13, 16])
def test_diagonal_pf_equals_binomial(n):
    ell = 2 * n + 1
    np.testing.assert_allclose(kl.rational_pf(XS, n, 0), kl.g_binomial(XS, ell), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_upper_diagonal_pf_equals_binomial(n):
    np.testing.assert_allclose(kl.rational_pf(XS, n, 1), kl.g_binomial(XS, 2 * n), rtol=1e-12, atol=1e-14)


def test_tanh_form_and_symmetries():
    x = np.linspace(-0.99, 0.99, 101)
    for ell in (3, 5, 9, 17, 33):
        np.testing.assert_allclose(kl.g_binomial(x, ell), kl.g_tanh(x, ell), rtol=1e-12, atol=1e-14)
    xp = np.logspace(-2, 2, 50)
    for n in (2, 4, 8):  # Eq. pade_symmetry
        np.testing.assert_allclose(kl.rational_pf(1 / xp, n, 0), 1 / kl.rational_pf(xp, n, 0), rtol=1e-12)
        np.testing.assert_allclose(kl.rational_pf(1 / xp, n, 1), kl.rational_pf(xp, n, 1), rtol=1e-12)


def test_tab1_tab2_polynomials(golden_dir):
    for line in _read(golden_dir, "kl_polynomials_tab1_tab2.txt"):
        s = " ".join(line).split("|")
        n = int(s[0])
        p = [float(c) for c in s[1].split()]
        q = [float(c) for c in s[2].split()]
        x2 = XS * XS
        f = XS * sum(c * x2 ** k for k, c in enumerate(p)) / sum(c * x2 ** k for k, c in enumerate(q))
        np.testing.assert_allclose(kl.rational_pf(XS, n, 0), f, rtol=1e-12, atol=1e-14)


def test_continued_fractions(golden_dir):
    for line in _read(golden_dir, "kl_continued_fractions.txt"):
        s = " ".join(line).split("|")
        n = int(s[0])
        a = [float(Fraction(t)) for t in s[1].split()]
        b = [float(Fraction(t)) for t in s[2].split()]
        y = XS * XS
        tail = y + b[-1]
        for k in range(len(a) - 1, 0, -1):
            tail = y + b[k - 1] - a[k] / tail
        f = XS / (2 * n + 1) * (1 + a[0] / tail)
        np.testing.assert_allclose(kl.rational_pf(XS, n, 0), f, rtol=1e-12, atol=1e-14)


def test_nesting_and_cascade_coefficients():
    # Eq. nesting: g_3(g_3(x)) = g_9(x) = f_44; g_3 o g_3 o g_3 = g_27 = f_{13,13}
    f11 = lambda x: kl.rational_pf(x, 1, 0)
    np.testing.assert_allclose(f11(f11(XS)), kl.rational_pf(XS, 4, 0), rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(f11(f11(f11(XS))), kl.rational_pf(XS, 13, 0), rtol=1e-11, atol=1e-14)
    # Sec. 8: f_44 coefficients 1/9, (0.229..., 0.0311...), (0.296..., 0.333...), ...
    c0, w, s = kl.kl_coeffs(4)
    assert c0 == pytest.approx(1 / 9)
    assert [round(v, 3) for v in w] == [0.229, 0.296, 0.538, 1.900]
    assert s[0] == pytest.approx(0.0311, abs=1e-4) and s[3] == pytest.approx(7.55, abs=5e-3)
    # Sec. 8: the smallest shift quoted for n = 4 and the n = 1 shift 1/3
    assert kl.kl_coeffs(1)[2][0] == pytest.approx(1 / 3, rel=1e-15)
    c0, w, s = kl.kl_coeffs(13)
    assert w[0] == pytest.approx(0.0743, abs=1e-4) and s[0] == pytest.approx(0.00339, abs=1e-5)
    assert w[-1] == pytest.approx(5.50, abs=5e-3) and s[-1] == pytest.approx(73.2, abs=0.05)


def test_tab4_wouldbe_zero_mode(golden_dir):
    mpmath.mp.dps = 250  # k = 2 reaches 1e-161: keep the cancellation exact
    for n, k, mant, ex in _read(golden_dir, "kl_wouldbe_zero_mode_tab4.txt"):
        n, k, mant, ex = int(n), int(k), float(mant), int(ex)
        ell = (2 * n + 1) ** k
        if k == 1:  # direct partial-fraction evaluation in FP64
            val = 1.0 + float(kl.rational_pf(-0.8, n, 0))
            assert val == pytest.approx(mant * 10.0 ** ex, rel=0.02)
        # iterate the binomial form of g_{2n+1} at high precision for k <= 2
        if k <= 2:
            x = mpmath.mpf(-0.8)
            for _ in range(k):
                a, b = (1 + x) ** (2 * n + 1), (1 - x) ** (2 * n + 1)
                x = (a - b) / (a + b)
            got = 1 + x
        else:  # 1 + g_l(-0.8) = 2 / (1 + 9^l) exactly (tanh form)
            got = 2 / (1 + mpmath.mpf(9) ** ell)
        # every printed entry is the correctly rounded value except n=5, k=1
        # (6.37e-11 printed as 6.3e-11): allow one unit in the last digit
        assert float(got / mpmath.mpf(10) ** ex) == pytest.approx(mant, abs=0.1)


def test_derivative_formula():
    x = np.linspace(-0.9, 0.9, 37)
    h = 1e-6
    for ell in (3, 9, 17):
        fd = (kl.g_binomial(x + h, ell) - kl.g_binomial(x - h, ell)) / (2 * h)
        np.testing.assert_allclose(kl.g_derivative(x, ell), fd, rtol=1e-7, atol=1e-9)
        assert np.all(kl.g_derivative(x, ell) >= 0)


def test_scale_parameter():
    for n in (4, 16):
        for s in (0.5, 3.0):
            np.testing.assert_allclose(kl.rational_pf(XS, n, 0, s), kl.rational_pf(XS / s, n, 0),
                                       rtol=1e-12, atol=1e-14)
