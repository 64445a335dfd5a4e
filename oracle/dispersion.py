"""Free-field quark dispersion relations (Sec. 2, App. A).

For a spatial momentum p = (p1, p2, p3) (a = 1) the energy E of the free
quark is the zero of the denominator of the free-field propagator after the
continuation p4 -> iE.  With the momentum-space forms of freefield.py
(evaluated at the complex momentum (p1, p2, p3, iE), where every term stays
real):

  kernel  K(p)^2 + M(p)^2 = 0,
          K = p_bar (Wilson) or p_tilde (Brillouin), M = p_hat^2/2 + m or
          p_check^2/2 + m;
  overlap (c^2 + d^2) [K^2 + M_-^2]^{1/2} + 2 c d M_- = 0,
          M_- = p_hat^2/2 - rho (or p_check^2/2 - rho), c = rho + m/2,
          d = rho - m/2 (the exact sign function of App. A).

The physical energy is the smallest positive root.  This module scans
cosh(E) upwards from 1 for the first sign change of the condition and refines
it with Brent's method (scipy.optimize.brentq).  TEST INFRASTRUCTURE ONLY
(see the package docstring).
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq

from .freefield import p_bar, p_check2, p_hat2, p_tilde


def _momentum(p, energy):
    return (complex(p[0]), complex(p[1]), complex(p[2]), 1j * energy)


def kernel_condition(energy, p, am, kind):
    """K^2 + M^2 at p4 = iE for the free Wilson ('wil') or Brillouin ('bri') operator."""
    q = _momentum(p, energy)
    if kind == "bri":
        k, mass = p_tilde(q), 0.5 * p_check2(q) + am
    else:
        k, mass = p_bar(q), 0.5 * p_hat2(q) + am
    val = np.sum(k * k) + mass * mass
    return float(np.real(val))


def overlap_condition(energy, p, am, rho, kind):
    """(c^2 + d^2) sqrt(K^2 + M_-^2) + 2 c d M_- at p4 = iE (exact overlap, App. A)."""
    q = _momentum(p, energy)
    if kind == "bri":
        k, mass = p_tilde(q), 0.5 * p_check2(q) - rho
    else:
        k, mass = p_bar(q), 0.5 * p_hat2(q) - rho
    k2 = float(np.real(np.sum(k * k)))
    mass = float(np.real(mass))
    c, d = rho + 0.5 * am, rho - 0.5 * am
    rad = k2 + mass * mass
    if rad < 0.0:
        return float("nan")
    return (c * c + d * d) * np.sqrt(rad) + 2.0 * c * d * mass


def energy(p, am, kind, overlap=False, rho=1.0, emax=8.0, nscan=4000):
    """Smallest positive E with a zero of the condition (nan if none below emax)."""
    if overlap:
        f = lambda e: overlap_condition(e, p, am, rho, kind)  # noqa: E731
    else:
        f = lambda e: kernel_condition(e, p, am, kind)  # noqa: E731
    # scan uniformly in E (the conditions are smooth in E); a zero at E = 0
    # itself (massless quark at rest) is returned as 0, also when rounding
    # leaves the condition a few ulps away from zero there
    grid = np.linspace(0.0, emax, nscan + 1)
    prev = f(grid[0])
    if abs(prev) <= 1e-12:
        return 0.0
    for a, b in zip(grid[:-1], grid[1:]):
        cur = f(b)
        if np.isfinite(prev) and np.isfinite(cur) and prev * cur <= 0.0:
            return brentq(f, a, b, xtol=1e-15, rtol=1e-15, maxiter=200)
        prev = cur
    return float("nan")
