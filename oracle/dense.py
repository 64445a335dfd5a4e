"""Dense matrices on tiny lattices (2^4, 4^4) and exact matrix functions.

Used to pin the Krylov-based oracle: the dense kernel matrix is assembled
column by column from the position-space operator, H = gamma5 D is
diagonalised with LAPACK (numpy.linalg.eigh) and f(H), sign(H) are formed as
V diag(f(lambda)) V^dagger (Sec. 5 uses the same full diagonalisation on small
lattices).
"""
from __future__ import annotations

import numpy as np

from .conventions import gammas


def dense_matrix(apply, site_shape, chunk=384):
    """Columns of the linear map ``apply`` on spinors x[rhs, t,z,y,x, 4, 3]."""
    nsite = int(np.prod(site_shape))
    dim = nsite * 12
    mat = np.zeros((dim, dim), dtype=np.complex128)
    for start in range(0, dim, chunk):
        stop = min(dim, start + chunk)
        e = np.zeros((stop - start, dim), dtype=np.complex128)
        e[np.arange(stop - start), np.arange(start, stop)] = 1.0
        cols = apply(e.reshape((stop - start,) + tuple(site_shape) + (4, 3)))
        mat[:, start:stop] = cols.reshape(stop - start, dim).T
    return mat


def gamma5_dense(nsite):
    _, g5 = gammas()
    return np.kron(np.eye(nsite), np.kron(g5, np.eye(3)))


def hermitian_function(h, func):
    lam, vec = np.linalg.eigh(h)
    return (vec * func(lam)) @ vec.conj().T, lam
