"""Off-axis parallel transporters W_d(n) by explicit path enumeration.

App. C (Brillouin operator flop count): within every k-hop contribution the
transporter is the average over the k! shortest lattice paths from n to n+d,
each the ordered product of the (smeared) links along it; the paper favours
this average over a back-projection to SU(3), so none is applied here.

A step +mu from site y uses U_mu(y); a step -mu from y uses U_mu(y-mu)^dagger.
This module enumerates every one of the 632 paths (80 offsets) literally; it
does not use any recursion, so it independently checks the level-by-level
construction of the CUDA library.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .conventions import all_offsets, dag, shift_by


def apply_time_bc(u, antiperiodic_t):
    """Antiperiodic time direction: flip the sign of U_t on the last slice."""
    if not antiperiodic_t:
        return u
    u = u.copy()
    u[-1, :, :, :, 3] *= -1.0
    return u


def path_product(u, path):
    """Product of links along ``path`` = [(mu, s), ...] starting at every n."""
    pos = [0, 0, 0, 0]
    prod = None
    for mu, s in path:
        if s > 0:
            step = shift_by(u[..., mu, :, :], tuple(pos))
        else:
            back = list(pos)
            back[mu] -= 1
            step = dag(shift_by(u[..., mu, :, :], tuple(back)))
        prod = step if prod is None else prod @ step
        pos[mu] += s
    return prod


def offaxis_links(u, antiperiodic_t=False):
    """W[idx, t, z, y, x, a, b] for all 81 offsets (idx 40 = identity)."""
    u = apply_time_bc(u, antiperiodic_t)
    site_shape = u.shape[:4]
    w = np.zeros((81,) + site_shape + (3, 3), dtype=np.complex128)
    for idx, d in enumerate(all_offsets()):
        dims = [mu for mu in range(4) if d[mu] != 0]
        if not dims:
            w[idx] = np.eye(3)
            continue
        acc = np.zeros(site_shape + (3, 3), dtype=np.complex128)
        for perm in itertools.permutations(dims):
            acc += path_product(u, [(mu, d[mu]) for mu in perm])
        w[idx] = acc / math.factorial(len(dims))
    return w


def stored_links(w):
    """The 40 stored links nu = 1..40 in the App. C layout [site][40][3][3]."""
    site_shape = w.shape[1:5]
    v = int(np.prod(site_shape))
    return np.ascontiguousarray(np.moveaxis(w[:40], 0, 4).reshape(v, 40, 3, 3))
