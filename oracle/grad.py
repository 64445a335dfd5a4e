"""Gradient of L = Re <eta, D_m psi> (sum over right-hand sides), FP64.

D_m = (1 - am/(2 rho)) D_ov + am with D_ov = rho (1 + D r(D^dagger D)),
r(s) = c0 + sum_i w_i / (s + sigma_i) (Eqs. def_over, KLnn_parfrac,
def_mass_traditional), D the Brillouin or Wilson kernel at m0 = -rho, with
or without the clover term (Eqs. def_bril, def_wils).
The real-gradient convention is dL = Re <g, d psi> and
dL = Re sum_{n,mu} tr(G_mu(n)^dagger dU_mu(n)) (the convention of PyTorch's
complex autograd).  The paper gives the ingredients (Sec. 9: with a
fixed-order rational the inner derivative is straightforward); the chain rule
written out here is:

  g_psi = D_m^dagger eta = gamma5 D_m gamma5 eta;
  with k = (1 - am/(2 rho)) rho, x_i = (A + sigma_i)^{-1} psi,
  z_i = (A + sigma_i)^{-1} D^dagger eta, y = c0 psi + sum_i w_i x_i:
  dL = k Re<eta, dD y> - k sum_i w_i [Re<D x_i, dD z_i> + Re<D z_i, dD x_i>],
  and Re<u, dD v> = Re sum_{n,d} tr(dW_d(n) F), F = sum_s (M_d v(n+d))_s u(n)_s^dagger,
  i.e. a gradient G_W = u (M_d v(n+d))^dagger for every transporter W_d(n).
  Each W_d(n) is the average over its k! paths of link products (App. C); a
  link U at position j of a path product A U B receives A^dagger G_W B^dagger
  (a backward step U^dagger receives B G_W^dagger A).  This module enumerates
  every path literally, independently of the recursion used on the GPU.

The clover term C(n) = -(c_SW/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(n),
F = P[(Q - Q^dagger)/(8i)] (P: traceless part, Q: the sum of the four leaves
around n in the (mu, nu) plane), contributes Re<u, dC v>, whose gradient with
respect to F_{mu nu}(n) is G_F = -(c_SW/2) sum_t (sigma_{mu nu} u(n))_t v_t(n)^dagger
(colour outer product, spin summed).  P is self-adjoint under Re tr(A^dagger B),
and Re tr(G^dagger (dQ - dQ^dagger)/(8i)) = Re tr(G_Q^dagger dQ) with
G_Q = (i/8) (P G_F + (P G_F)^dagger); G_Q then flows into the links of every
leaf with the same rule as for a path product.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .conventions import all_offsets, dag, gammas, shift_by
from .dirac import DiracOperator, gamma5
from .kl import kl_coeffs
from .links import apply_time_bc
from .mscg import multishift_cg
from .overlap import overlap_apply


def _shift_back(f, d):
    """Move a per-site quantity defined at n to the site n + d (inverse of shift_by)."""
    return shift_by(f, tuple(-c for c in d))


def transporter_gradient(kernel, pairs):
    """G_W[idx] (per offset, per site) from sum_p weight_p Re<u_p, dD v_p>.

    pairs: list of (u[rhs=1,...], v[rhs=1,...], weight).
    """
    site_shape = kernel.w.shape[1:5]
    gw = np.zeros((81,) + site_shape + (3, 3), dtype=np.complex128)
    for idx, d in enumerate(all_offsets()):
        if idx == 40:
            continue
        m = kernel.mats[idx]
        for u, v, wt in pairs:
            vs = shift_by(v[0], d)                               # v(n + d)
            chi = np.einsum("st,...ta->...sa", m, vs)             # M_d v(n+d)
            gw[idx] += wt * np.einsum("...sa,...sb->...ab", u[0], chi.conj())
    return gw


def link_gradient_from_transporters(u_bc, gw):
    """G_U[t,z,y,x,mu,3,3] from the transporter gradients by path enumeration."""
    site_shape = u_bc.shape[:4]
    gu = np.zeros(site_shape + (4, 3, 3), dtype=np.complex128)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), site_shape + (3, 3))
    for idx, d in enumerate(all_offsets()):
        dims = [mu for mu in range(4) if d[mu] != 0]
        if not dims:
            continue
        scale = 1.0 / math.factorial(len(dims))
        for perm in itertools.permutations(dims):
            # the steps of this path, with the site (relative to n) of each link
            steps = []
            pos = [0, 0, 0, 0]
            for mu in perm:
                s = d[mu]
                if s > 0:
                    steps.append((mu, +1, tuple(pos)))
                else:
                    back = list(pos)
                    back[mu] -= 1
                    steps.append((mu, -1, tuple(back)))
                pos[mu] += s
            mats = []
            for mu, s, at in steps:
                link = shift_by(u_bc[..., mu, :, :], at)
                mats.append(link if s > 0 else dag(link))
            for j, (mu, s, at) in enumerate(steps):
                a = eye
                for mm in mats[:j]:
                    a = a @ mm
                b = eye
                for mm in mats[j + 1:]:
                    b = b @ mm
                if s > 0:
                    contrib = dag(a) @ gw[idx] @ dag(b)
                else:
                    contrib = b @ dag(gw[idx]) @ a
                gu[..., mu, :, :] += scale * _shift_back(contrib, at)
    return gu


def _clover_leaves(mu, nu):
    """The four leaves at n in the (mu, nu) plane, each as its four factors
    (direction, daggered, site offset a e_mu + b e_nu), in product order."""
    def at(a, b):
        return tuple(a * (k == mu) + b * (k == nu) for k in range(4))
    return [
        [(mu, False, at(0, 0)), (nu, False, at(1, 0)), (mu, True, at(0, 1)), (nu, True, at(0, 0))],
        [(nu, False, at(0, 0)), (mu, True, at(-1, 1)), (nu, True, at(-1, 0)), (mu, False, at(-1, 0))],
        [(mu, True, at(-1, 0)), (nu, True, at(-1, -1)), (mu, False, at(-1, -1)), (nu, False, at(0, -1))],
        [(nu, True, at(0, -1)), (mu, False, at(0, -1)), (nu, False, at(1, -1)), (mu, True, at(0, 0))],
    ]


def clover_link_gradient(u_bc, c_sw, pairs):
    """G_U[t,z,y,x,mu,3,3] of sum_p weight_p Re<u_p, dC v_p> (clover term only)."""
    g, _ = gammas()
    site_shape = u_bc.shape[:4]
    gu = np.zeros(site_shape + (4, 3, 3), dtype=np.complex128)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), site_shape + (3, 3))
    for mu in range(4):
        for nu in range(mu + 1, 4):
            sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            gf = np.zeros(site_shape + (3, 3), dtype=np.complex128)
            for u, v, wt in pairs:
                su = np.einsum("ts,...sa->...ta", sig, u[0])
                gf += -0.5 * c_sw * wt * np.einsum("...ta,...tb->...ab", su, v[0].conj())
            gp = gf - np.trace(gf, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
            gq = 0.125j * (gp + dag(gp))
            for leaf in _clover_leaves(mu, nu):
                mats = []
                for d, is_dag, at in leaf:
                    link = shift_by(u_bc[..., d, :, :], at)
                    mats.append(dag(link) if is_dag else link)
                for j, (d, is_dag, at) in enumerate(leaf):
                    a = eye
                    for mm in mats[:j]:
                        a = a @ mm
                    b = eye
                    for mm in mats[j + 1:]:
                        b = b @ mm
                    contrib = b @ dag(gq) @ a if is_dag else dag(a) @ gq @ dag(b)
                    gu[..., d, :, :] += _shift_back(contrib, at)
    return gu


def overlap_grad(u, eta, psi, rho, n, tol, am=0.0, kind=0, antiperiodic_t=False, c_sw=0.0, kernel="bri"):
    """(g_psi, G_U) for L = Re <eta, D_m psi> summed over the right-hand sides."""
    kern = DiracOperator(u, kernel, m0=-rho, c_sw=c_sw, antiperiodic_t=antiperiodic_t)
    g_psi, _ = overlap_apply(kern, gamma5(eta), rho, n, tol, am=am, kind=kind)
    g_psi = gamma5(g_psi)
    c0, w, sig = kl_coeffs(n, kind)
    k = (1.0 - am / (2.0 * rho)) * rho
    pairs = []
    for r in range(psi.shape[0]):
        p, e = psi[r:r + 1], eta[r:r + 1]
        xs, _ = multishift_cg(kern.normal, p, sig, tol)
        zs, _ = multishift_cg(kern.normal, kern.apply_dagger(e), sig, tol)
        y = c0 * p
        for wi, xi in zip(w, xs):
            y = y + wi * xi
        pairs.append((e, y, k))
        for wi, xi, zi in zip(w, xs, zs):
            pairs.append((kern.apply(xi), zi, -k * wi))
            pairs.append((kern.apply(zi), xi, -k * wi))
    gw = transporter_gradient(kern, pairs)
    u_bc = apply_time_bc(u, antiperiodic_t)
    gu = link_gradient_from_transporters(u_bc, gw)
    if c_sw != 0.0:
        gu = gu + clover_link_gradient(u_bc, c_sw, pairs)
    if antiperiodic_t:
        gu[-1, :, :, :, 3] *= -1.0
    return g_psi, gu


def loss(u, eta, psi, rho, n, tol, am=0.0, kind=0, antiperiodic_t=False, c_sw=0.0, kernel="bri"):
    kern = DiracOperator(u, kernel, m0=-rho, c_sw=c_sw, antiperiodic_t=antiperiodic_t)
    y, _ = overlap_apply(kern, psi, rho, n, tol, am=am, kind=kind)
    return float(np.vdot(eta.ravel(), y.ravel()).real)
