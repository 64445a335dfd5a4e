"""Kenney-Laub rational approximations to sign(x) (Sec. 3, App. B).

* principal Pade iteration functions g_l (Eq. def_gell), the binomial form
  ((1+x)^l - (1-x)^l) / ((1+x)^l + (1-x)^l) and the tanh(l artanh x) form;
* diagonal f_nn = g_{2n+1} in partial fractions (Eq. KLnn_parfrac):
    g_{2n+1}(x) = x/(2n+1) sum_{i=0}^{n} (2 - delta_{i,n})
                  / (sin^2 theta_i + cos^2 theta_i x^2),
    theta_i = (2i+1) pi / (4n+2);
  the i = n term is the constant 1, the others become w_i / (x^2 + sigma_i)
  with sigma_i = tan^2 theta_i and w_i = 2 / ((2n+1) cos^2 theta_i);
* upper diagonal g_{2n} (Sec. 3.3): (x/n) sum_{i<n} 1/(sin^2 + cos^2 x^2),
  theta_i = (2i+1) pi/(4n): sigma_i = tan^2 theta_i, w_i = 1/(n cos^2 theta_i);
* an optional spectral scale s: f(x/s) = x [c0/s + sum (w_i s)/(x^2 + sigma_i s^2)].
"""
from __future__ import annotations

import math

import numpy as np


def kl_coeffs(n, kind=0, scale=1.0):
    """(c0, w[n], sigma[n]) with f(x) = x (c0 + sum_i w_i / (x^2 + sigma_i)).

    kind 0: diagonal f_nn = g_{2n+1}; kind 1: upper diagonal g_{2n}.
    Shifts are returned in increasing order.
    """
    n = int(n)
    if n < 1:
        raise ValueError("order n must be >= 1")
    s = float(scale)
    w = np.zeros(n)
    sig = np.zeros(n)
    if kind == 0:
        for i in range(n):
            th = (2 * i + 1) * math.pi / (4 * n + 2)
            sig[i] = math.tan(th) ** 2
            w[i] = 2.0 / ((2 * n + 1) * math.cos(th) ** 2)
        c0 = 1.0 / (2 * n + 1)
    elif kind == 1:
        for i in range(n):
            th = (2 * i + 1) * math.pi / (4 * n)
            sig[i] = math.tan(th) ** 2
            w[i] = 1.0 / (n * math.cos(th) ** 2)
        c0 = 0.0
    else:
        raise ValueError("kind must be 0 (diagonal) or 1 (upper diagonal)")
    return c0 / s, w * s, sig * s * s


def rational_pf(x, n, kind=0, scale=1.0):
    """x (c0 + sum w_i/(x^2+sigma_i)), the partial-fraction evaluation."""
    c0, w, sig = kl_coeffs(n, kind, scale)
    x = np.asarray(x, dtype=np.float64)
    return x * (c0 + sum(w[i] / (x * x + sig[i]) for i in range(len(w))))


def rational_r(y, n, kind=0, scale=1.0):
    """r(y) = c0 + sum w_i / (y + sigma_i), so that f(x) = x r(x^2)."""
    c0, w, sig = kl_coeffs(n, kind, scale)
    return c0 + sum(w[i] / (y + sig[i]) for i in range(len(w)))


def g_binomial(x, ell):
    """Eq. def_gell."""
    x = np.asarray(x, dtype=np.float64)
    a, b = (1 + x) ** ell, (1 - x) ** ell
    return (a - b) / (a + b)


def g_tanh(x, ell):
    """g_l(x) = tanh(l artanh x) for |x| < 1."""
    return np.tanh(ell * np.arctanh(np.asarray(x, dtype=np.float64)))


def g_derivative(x, ell):
    """g_l'(x) = 4 l (1-x^2)^(l-1) / [(1+x)^l + (1-x)^l]^2 (Sec. 9)."""
    x = np.asarray(x, dtype=np.float64)
    return 4 * ell * (1 - x * x) ** (ell - 1) / ((1 + x) ** ell + (1 - x) ** ell) ** 2
