"""Wilson and Brillouin Dirac operators in position space (FP64).

Eqs. def_wils / def_bril (Sec. 1):
  D = sum_mu gamma_mu nabla_mu - (1/2) Delta + m0 - (c_SW/2) sum_{mu<nu} sigma_{mu nu} F_{mu nu}
with a = 1.  The stencil weights are obtained by expanding the momentum-space
definitions of App. A into plane waves: a symbol f(p) = sum_d c_d e^{i p.d}
acts as (f x)(n) = sum_d c_d x(n+d).  Per dimension
  i sin p   -> {+1: +1/2, -1: -1/2}
  cos p + 2 -> {+1: 1/2, 0: 2, -1: 1/2}
  cos p + 1 -> {+1: 1/2, 0: 1, -1: 1/2}
  2 cos p - 2 -> {+1: 1, 0: -2, -1: 1}
and
  nabla^std_mu = i sin p_mu,
  nabla^iso_mu = (i/27) sin p_mu prod_{nu != mu} (cos p_nu + 2),
  Delta^std    = sum_mu (2 cos p_mu - 2),
  Delta^bri    = (1/4) prod_mu (cos p_mu + 1) - 4.
Each offset d is gauged with the path-averaged transporter W_d(n) (App. C).

Clover (the paper leaves sigma and F undefined): F_{mu nu} is the
anti-Hermitian part of the four-leaf clover Q_{mu nu}, F = (Q - Q^dag)/(8i),
made traceless, and sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu].
"""
from __future__ import annotations

import numpy as np

from .conventions import all_offsets, dag, gammas, shift

_ISIN = {1: 0.5, -1: -0.5, 0: 0.0}
_COS2 = {1: 0.5, 0: 2.0, -1: 0.5}
_COS1 = {1: 0.5, 0: 1.0, -1: 0.5}
_LAPSTD = {1: 1.0, 0: -2.0, -1: 1.0}


def nabla_iso_weight(d, mu):
    """Position-space weight of nabla^iso_mu at offset d (App. A)."""
    w = _ISIN[d[mu]] / 27.0
    for nu in range(4):
        if nu != mu:
            w *= _COS2[d[nu]]
    return w


def lap_bri_weight(d):
    """Position-space weight of Delta^bri at offset d (App. A)."""
    w = 0.25
    for mu in range(4):
        w *= _COS1[d[mu]]
    if d == (0, 0, 0, 0):
        w -= 4.0
    return w


def nabla_std_weight(d, mu):
    if any(d[nu] != 0 for nu in range(4) if nu != mu):
        return 0.0
    return _ISIN[d[mu]]


def lap_std_weight(d):
    nz = [mu for mu in range(4) if d[mu] != 0]
    if len(nz) > 1:
        return 0.0
    if len(nz) == 1:
        return _LAPSTD[d[nz[0]]]
    return sum(_LAPSTD[0] for _ in range(4))


def spin_matrices(kind, m0):
    """81 spin matrices M_d with D = sum_d M_d W_d(n) x(n+d) (clover aside)."""
    g, _ = gammas()
    mats = np.zeros((81, 4, 4), dtype=np.complex128)
    for idx, d in enumerate(all_offsets()):
        if kind == "bri":
            m = sum(nabla_iso_weight(d, mu) * g[mu] for mu in range(4))
            m = m - 0.5 * lap_bri_weight(d) * np.eye(4)
        elif kind == "wil":
            m = sum(nabla_std_weight(d, mu) * g[mu] for mu in range(4))
            m = m - 0.5 * lap_std_weight(d) * np.eye(4)
        else:
            raise ValueError(kind)
        if idx == 40:
            m = m + m0 * np.eye(4)
        mats[idx] = m
    return mats


def clover_field(u, c_sw):
    """Per-site 12x12 clover matrix -(c_SW/2) sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}.

    Returned as C[t,z,y,x, s, a, s', b] (spin s, colour a).
    """
    g, _ = gammas()
    site_shape = u.shape[:4]
    c = np.zeros(site_shape + (4, 3, 4, 3), dtype=np.complex128)
    if c_sw == 0.0:
        return c
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um, un = u[..., mu, :, :], u[..., nu, :, :]
            # four leaves of the clover around n in the (mu, nu) plane
            l1 = um @ shift(un, mu, 1) @ dag(shift(um, nu, 1)) @ dag(un)
            un_mm = shift(un, mu, -1)
            um_mm = shift(um, mu, -1)
            l2 = un @ dag(shift(shift(um, mu, -1), nu, 1)) @ dag(un_mm) @ um_mm
            l3 = (dag(um_mm) @ dag(shift(shift(un, mu, -1), nu, -1))
                  @ shift(shift(um, mu, -1), nu, -1) @ shift(un, nu, -1))
            un_nm = shift(un, nu, -1)
            l4 = dag(un_nm) @ shift(um, nu, -1) @ shift(shift(un, nu, -1), mu, 1) @ dag(um)
            q = l1 + l2 + l3 + l4
            f = (q - dag(q)) / 8j
            f = f - np.trace(f, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3.0
            sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
            c += -0.5 * c_sw * np.einsum("st,...ab->...satb", sig, f)
    return c


def apply_stencil(w, mats, x, clover=None):
    """y(n) = sum_d M_d W_d(n) x(n+d) [+ C(n) x(n)] for x[rhs,t,z,y,x,4,3]."""
    y = np.zeros_like(x)
    for idx, d in enumerate(all_offsets()):
        m = mats[idx]
        if not np.any(m):
            continue
        xs = x
        for mu in range(4):
            if d[mu]:
                xs = shift(xs, mu, d[mu], lead=1)
        wx = np.swapaxes(w[idx] @ np.swapaxes(xs, -1, -2), -1, -2)  # colour
        y += np.einsum("st,...ta->...sa", m, wx)                     # spin
    if clover is not None:
        y += np.einsum("...satb,r...tb->r...sa", clover, x)
    return y


def gamma5(x):
    _, g5 = gammas()
    return np.einsum("st,...ta->...sa", g5, x)


class DiracOperator:
    """D_bri or D_wil at bare mass m0 on a fixed gauge background (FP64)."""

    def __init__(self, u, kind="bri", m0=0.0, c_sw=0.0, antiperiodic_t=False, w=None):
        from .links import apply_time_bc, offaxis_links
        self.kind = kind
        self.m0 = float(m0)
        ub = apply_time_bc(u, antiperiodic_t)
        if kind == "bri":
            self.w = offaxis_links(u, antiperiodic_t) if w is None else w
        else:
            self.w = self._wilson_links(ub)
        self.mats = spin_matrices(kind, m0)
        self.clover = clover_field(ub, c_sw) if c_sw != 0.0 else None

    @staticmethod
    def _wilson_links(u):
        site_shape = u.shape[:4]
        w = np.zeros((81,) + site_shape + (3, 3), dtype=np.complex128)
        w[40] = np.eye(3)
        for mu in range(4):
            e = [0, 0, 0, 0]
            e[mu] = 1
            fwd = (e[0] + 1) + 3 * (e[1] + 1) + 9 * (e[2] + 1) + 27 * (e[3] + 1)
            w[fwd] = u[..., mu, :, :]
            w[80 - fwd] = dag(shift(u[..., mu, :, :], mu, -1))
        return w

    def apply(self, x):
        return apply_stencil(self.w, self.mats, x, self.clover)

    def apply_dagger(self, x):
        """D^dagger = gamma5 D gamma5 (gamma5-hermiticity, Eq. def_over)."""
        return gamma5(self.apply(gamma5(x)))

    def normal(self, x):
        """A = D^dagger D."""
        return self.apply_dagger(self.apply(x))


def _site_links_walk(u, site, d):
    """W_d at one site by walking every shortest path with explicit coordinates."""
    import itertools
    import math
    lt, lz, ly, lx = u.shape[:4]
    dims = (lx, ly, lz, lt)

    def link(pos, mu):
        return u[pos[3] % lt, pos[2] % lz, pos[1] % ly, pos[0] % lx, mu]

    nz = [mu for mu in range(4) if d[mu] != 0]
    acc = np.zeros((3, 3), dtype=np.complex128)
    for perm in itertools.permutations(nz):
        pos = list(site)
        prod = np.eye(3, dtype=np.complex128)
        for mu in perm:
            if d[mu] > 0:
                prod = prod @ link(pos, mu)
                pos[mu] += 1
            else:
                pos[mu] -= 1
                prod = prod @ link(pos, mu).conj().T
        acc += prod
    return acc / math.factorial(len(nz)), dims


def apply_at_sites(u, kind, m0, c_sw, x, sites, antiperiodic_t=False):
    """y(n) = (D x)(n) at the listed sites only (x[rhs, t,z,y,x, 4, 3]).

    A per-site restatement for sampled checks on lattices too large for the
    whole-field oracle: transporters by explicit path walks, the clover term
    from the four leaves at that site, the same stencil weights.
    """
    from .links import apply_time_bc
    ub = apply_time_bc(u, antiperiodic_t)
    lt, lz, ly, lx = ub.shape[:4]
    mats = spin_matrices(kind, m0)
    out = np.zeros((x.shape[0], len(sites), 4, 3), dtype=np.complex128)
    g, _ = gammas()
    for i, site in enumerate(sites):
        sx, sy, sz, st = site
        for idx, d in enumerate(all_offsets()):
            m = mats[idx]
            if not np.any(m):
                continue
            if idx == 40:
                w = np.eye(3)
            elif kind == "bri":
                w, _ = _site_links_walk(ub, site, d)
            else:
                mu = [k for k in range(4) if d[k] != 0][0]
                if d[mu] > 0:
                    w = ub[st, sz, sy, sx, mu]
                else:
                    p = list(site)
                    p[mu] -= 1
                    w = ub[p[3] % lt, p[2] % lz, p[1] % ly, p[0] % lx, mu].conj().T
            xs = x[:, (st + d[3]) % lt, (sz + d[2]) % lz, (sy + d[1]) % ly, (sx + d[0]) % lx]
            out[:, i] += np.einsum("st,ab,rtb->rsa", m, w, xs)
        if c_sw != 0.0:
            cl = np.zeros((4, 3, 4, 3), dtype=np.complex128)

            def L(pos, mu):
                return ub[pos[3] % lt, pos[2] % lz, pos[1] % ly, pos[0] % lx, mu]

            for mu in range(4):
                for nu in range(mu + 1, 4):
                    em = [int(k == mu) for k in range(4)]
                    en = [int(k == nu) for k in range(4)]
                    at = lambda a, b: [site[k] + a * em[k] + b * en[k] for k in range(4)]
                    q = (L(at(0, 0), mu) @ L(at(1, 0), nu) @ L(at(0, 1), mu).conj().T @ L(at(0, 0), nu).conj().T
                         + L(at(0, 0), nu) @ L(at(-1, 1), mu).conj().T @ L(at(-1, 0), nu).conj().T @ L(at(-1, 0), mu)
                         + L(at(-1, 0), mu).conj().T @ L(at(-1, -1), nu).conj().T @ L(at(-1, -1), mu)
                         @ L(at(0, -1), nu)
                         + L(at(0, -1), nu).conj().T @ L(at(0, -1), mu) @ L(at(1, -1), nu) @ L(at(0, 0), mu).conj().T)
                    f = (q - q.conj().T) / 8j
                    f = f - np.trace(f) * np.eye(3) / 3.0
                    sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
                    cl += -0.5 * c_sw * np.einsum("st,ab->satb", sig, f)
            out[:, i] += np.einsum("satb,rtb->rsa", cl, x[:, st, sz, sy, sx])
    return out
