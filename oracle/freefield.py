"""Free-field (U = 1) momentum-space forms of App. A.

  p_hat_mu = 2 sin(p_mu/2),  p_bar_mu = sin p_mu,
  p_tilde_mu = (1/27) sin p_mu prod_{nu != mu} (cos p_nu + 2),
  Delta^std = -p_hat^2,  Delta^bri = (1/4) prod_mu (cos p_mu + 1) - 4 = -p_check^2,
  D_W(p) = i p_bar.gamma + p_hat^2/2 + m,   D_B(p) = i p_tilde.gamma + p_check^2/2 + m,
  D^dagger D = p^2 + M^2 (a multiple of the identity), so the overlap of
  App. A becomes rho [1 + D_{-rho}(p) r(p^2 + M^2)] with the rational r
  standing in for [.]^{-1/2}.
"""
from __future__ import annotations

import numpy as np

from .conventions import gammas


def p_hat2(p):
    return sum((2 * np.sin(pm / 2)) ** 2 for pm in p)


def p_bar(p):
    return np.array([np.sin(pm) for pm in p])


def p_tilde(p):
    out = []
    for mu in range(4):
        v = np.sin(p[mu]) / 27.0
        for nu in range(4):
            if nu != mu:
                v *= np.cos(p[nu]) + 2.0
        out.append(v)
    return np.array(out)


def p_check2(p):
    return 4.0 - 0.25 * np.prod([np.cos(pm) + 1.0 for pm in p])


def kernel_symbol(p, kind, m0):
    """4x4 spin matrix D(p) of the free Wilson ('wil') or Brillouin ('bri') kernel."""
    g, _ = gammas()
    if kind == "bri":
        k, mass = p_tilde(p), 0.5 * p_check2(p) + m0
    else:
        k, mass = p_bar(p), 0.5 * p_hat2(p) + m0
    return 1j * sum(k[mu] * g[mu] for mu in range(4)) + mass * np.eye(4), float(np.dot(k, k)), mass


def overlap_symbol(p, kind, rho, r_of_y):
    """rho [1 + D_{-rho}(p) r(D^dag D)] for the free field."""
    d, k2, mass = kernel_symbol(p, kind, -rho)
    return rho * (np.eye(4) + d * r_of_y(k2 + mass * mass))
