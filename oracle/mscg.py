"""Multi-shift conjugate gradient (Sec. 3.3; App. B; Sec. 8).

Solves (A + sigma_i) x_i = b for all shifts in one Krylov space, A Hermitian
positive definite (here A = D^dagger D).  The base system is the smallest
shift sigma_0; the shifted residuals stay collinear with the base residual,
r_i = zeta_i r, and the recurrences follow from matching the three-term
Lanczos recurrence of CG for A + sigma_0 and for A + sigma_i
(delta_i = sigma_i - sigma_0):

  zeta_{k+1} = zeta_k zeta_{k-1} alpha_{k-1}
               / [alpha_k beta_{k-1} (zeta_{k-1} - zeta_k)
                  + zeta_{k-1} alpha_{k-1} (1 + delta alpha_k)]
  alpha^i_k = alpha_k zeta_{k+1} / zeta_k
  beta^i_k  = beta_k (zeta_{k+1} / zeta_k)^2
  x_i += alpha^i_k p_i ;  p_i = zeta_{k+1} r_{k+1} + beta^i_k p_i

with zeta_{-1} = zeta_0 = 1, alpha_{-1} = 1, beta_{-1} = 0.  A shift stops
(its x_i, p_i are frozen) once |zeta_i| ||r|| <= tol ||b||.
"""
from __future__ import annotations

import numpy as np


def vdot(a, b):
    return np.vdot(a.ravel(), b.ravel())


def multishift_cg(apply_a, b, sigmas, tol, maxiter=100000):
    """Return (x[n_shift], iterations) for one right-hand side b."""
    sig = np.asarray(sigmas, dtype=np.float64)
    order = np.argsort(sig)
    if not np.all(order == np.arange(len(sig))):
        raise ValueError("shifts must be sorted in increasing order")
    base = sig[0]
    delta = sig - base
    n = len(sig)
    x = [np.zeros_like(b) for _ in range(n)]
    p = [b.copy() for _ in range(n)]
    r = b.copy()
    rr = vdot(r, r).real
    bnorm = np.sqrt(rr)
    if bnorm == 0.0:
        return x, 0
    zeta = np.ones(n)
    zeta_prev = np.ones(n)
    alpha_prev, beta_prev = 1.0, 0.0
    active = np.ones(n, dtype=bool)
    it = 0
    for it in range(1, maxiter + 1):
        q = apply_a(p[0]) + base * p[0]
        alpha = rr / vdot(p[0], q).real
        zeta_next = zeta.copy()  # frozen shifts keep their last value
        for i in range(n):
            if not active[i]:
                continue
            den = (alpha * beta_prev * (zeta_prev[i] - zeta[i])
                   + zeta_prev[i] * alpha_prev * (1.0 + delta[i] * alpha))
            zeta_next[i] = zeta[i] * zeta_prev[i] * alpha_prev / den
        for i in range(n):
            if active[i]:
                x[i] = x[i] + (alpha * zeta_next[i] / zeta[i]) * p[i]
        r = r - alpha * q
        rr_new = vdot(r, r).real
        beta = rr_new / rr
        for i in range(n):
            if active[i]:
                beta_i = beta * (zeta_next[i] / zeta[i]) ** 2
                p[i] = zeta_next[i] * r + beta_i * p[i]
        zeta_prev, zeta = zeta, zeta_next
        alpha_prev, beta_prev, rr = alpha, beta, rr_new
        for i in range(n):
            if active[i] and abs(zeta[i]) * np.sqrt(rr) <= tol * bnorm:
                active[i] = False
        if not active.any():
            break
    return x, it


def true_residuals(apply_a, b, sigmas, x):
    """||b - (A + sigma_i) x_i|| / ||b|| for every shift (the absolute norm for a zero source)."""
    bn = np.sqrt(vdot(b, b).real)
    bn = bn if bn > 0.0 else 1.0
    return [np.sqrt(vdot(res, res).real) / bn
            for res in (b - apply_a(xi) - s * xi for xi, s in zip(x, sigmas))]
