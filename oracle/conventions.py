"""Lattice and spin conventions of the oracle (a = 1).

* site index n = x + Lx*(y + Ly*(z + Lz*t)); numpy field axes (t, z, y, x);
* mu = 0..3 <-> x, y, z, t;
* chiral (Weyl) basis, which App. C assumes when it counts the gamma
  right-multiplications as free permutations: gamma_k = [[0, -i s_k], [i s_k, 0]]
  (s_k the Pauli matrices), gamma_4 = [[0, 1], [1, 0]], so that
  gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1);
* the 81 hypercube offsets d in {-1,0,1}^4 are numbered (App. C) so that nu
  and 82-nu are opposite and nu = 41 is the zero hop:
  nu - 1 = (d_x+1) + 3 (d_y+1) + 9 (d_z+1) + 27 (d_t+1).
  nu = 1..40 are the stored links; their most significant (t first) nonzero
  component is -1.
"""
from __future__ import annotations

import itertools

import numpy as np


def shift(f, mu, s, lead=0):
    """Field at n + s*e_mu (periodic).  ``lead`` leading non-site axes."""
    return np.roll(f, -s, axis=lead + 3 - mu)


def shift_by(f, d, lead=0):
    """Field at n + d for an offset d = (dx, dy, dz, dt)."""
    out = f
    for mu in range(4):
        if d[mu]:
            out = shift(out, mu, d[mu], lead)
    return out


def dag(m):
    return np.swapaxes(m, -1, -2).conj()


def pauli():
    return np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128)


def gammas():
    """gamma_1..gamma_4 (index 0..3) in the chiral basis, and gamma_5."""
    s = pauli()
    z = np.zeros((2, 2), dtype=np.complex128)
    one = np.eye(2, dtype=np.complex128)
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    for k in range(3):
        g[k] = np.block([[z, -1j * s[k]], [1j * s[k], z]])
    g[3] = np.block([[z, one], [one, z]])
    g5 = g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


def nu_index(d):
    """0-based index nu-1 of offset d (App. C numbering)."""
    return (d[0] + 1) + 3 * (d[1] + 1) + 9 * (d[2] + 1) + 27 * (d[3] + 1)


def offset_of(idx):
    """Offset d for the 0-based index idx = nu - 1."""
    return (idx % 3 - 1, (idx // 3) % 3 - 1, (idx // 9) % 3 - 1, (idx // 27) % 3 - 1)


def all_offsets():
    """All 81 offsets in numbering order (index 40 is the zero hop)."""
    return [offset_of(i) for i in range(81)]


def hops(d):
    return sum(1 for c in d if c != 0)


def stored_offsets():
    """The 40 stored offsets nu = 1..40 (indices 0..39)."""
    return [offset_of(i) for i in range(40)]


def lattice_momenta(dims):
    """All periodic momenta p_mu = 2 pi k_mu / L_mu, as (Lx,Ly,Lz,Lt) tuples."""
    ranges = [range(int(L)) for L in dims]
    for k in itertools.product(*ranges):
        yield tuple(2 * np.pi * k[m] / dims[m] for m in range(4))
