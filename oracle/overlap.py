"""Overlap operator with a Kenney-Laub sign function (Sec. 4).

Eq. def_over with a = 1:  D_ov = rho [1 + gamma5 sign(H)],  H = gamma5 D_{-rho},
for a gamma5-hermitian kernel D_{-rho} (bare mass m0 = -rho).  The sign
function is replaced by the diagonal Kenney-Laub rational f_nn(x) =
x r(x^2), r(y) = c0 + sum_i w_i/(y + sigma_i) (Eq. KLnn_parfrac).  Since
H^2 = D^dagger D and gamma5 H = D, Sec. 4.1 reduces everything to products
with D^dagger D and D:

  gamma5 f(H) b = D r(D^dagger D) b = D (c0 b + sum_i w_i x_i),
  x_i = (D^dagger D + sigma_i)^{-1} b   (one multi-shift CG solve).

Massive forms (Sec. 4.2, 4.3):
  traditional  D_m = (1 - am/(2 rho)) D_ov + am            (Eq. def_mass_traditional)
  complete     solve (D_ov + mt) x = bt with mt = am/(1 - am/(2 rho)) and
               bt = [1 + am/(2 rho) (1 - D_ov/(2 rho))] b / (1 - am/(2 rho))
                                                            (Eq. upshot_complete)
"""
from __future__ import annotations

import numpy as np

from .kl import kl_coeffs
from .mscg import multishift_cg, true_residuals


def sign_apply(kernel, b, n, tol, scale=1.0, kind=0, maxiter=100000):
    """gamma5 f_nn(H) b for every rhs in b[rhs, ...]; kernel at m0 = -rho.

    Returns (y, info) with info = per-rhs dict(iterations, residuals).
    """
    c0, w, sig = kl_coeffs(n, kind, scale)
    y = np.zeros_like(b)
    info = []
    for r in range(b.shape[0]):
        br = b[r:r + 1]
        xs, it = multishift_cg(kernel.normal, br, sig, tol, maxiter)
        acc = c0 * br
        for wi, xi in zip(w, xs):
            acc = acc + wi * xi
        y[r:r + 1] = kernel.apply(acc)
        info.append(dict(iterations=it, residuals=true_residuals(kernel.normal, br, sig, xs)))
    return y, info


def overlap_apply(kernel, b, rho, n, tol, am=0.0, scale=1.0, kind=0, maxiter=100000):
    """(1 - am/(2 rho)) rho (b + gamma5 f(H) b) + am b  (am = 0: massless)."""
    s, info = sign_apply(kernel, b, n, tol, scale, kind, maxiter)
    dov = rho * (b + s)
    return (1.0 - am / (2.0 * rho)) * dov + am * b, info


def complete_mass_rhs(dov_b, b, rho, am):
    """(mt, bt) of Eq. upshot_complete, given dov_b = D_ov b (massless)."""
    k = 1.0 - am / (2.0 * rho)
    mt = am / k
    bt = (b + (am / (2.0 * rho)) * (b - dov_b / (2.0 * rho))) / k
    return mt, bt


def traditional_mass_rhs(b, rho, am):
    """(mt, bt) of Eq. upshot_traditional."""
    k = 1.0 - am / (2.0 * rho)
    return am / k, b / k
