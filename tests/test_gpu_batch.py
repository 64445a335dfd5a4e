"""Batched overlap application over independent lattices of uneven volume
(concurrent streams, graph-replayed solver iterations, autotuned stencil):
every lattice against the FP64 oracle, FP64 within 1e-12 and the mixed path
within 1e-10, and identical results to per-lattice calls.  Lattice 0 carries
the 12 spin-colour point sources."""
import functools

import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, overlap
from paper_1701_00726_gb300 import PREC_F32, PREC_F64, Lattice, overlap_apply_batch

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 4, 2), (4, 4, 2, 6), (2, 2, 2, 8)]
ORDER = 12


def relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _inputs(i, dims):
    """Lattice 0: the 12 point sources (six two-rhs work items); lattice 1: three sources (one
    two-rhs item and a single); the others one source each (single items)."""
    u = sf.gauge_field(dims, 20 + i, 0.1, 3)
    src = sf.point_sources(dims) if i == 0 else sf.gaussian_source(dims, 3 if i == 1 else 1, 40 + i)
    return u, src


@functools.lru_cache(maxsize=None)
def _oracle(i):
    u, src = _inputs(i, SHAPES[i])
    want, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), src, 1.0, ORDER, 1e-13)
    return want


@pytest.mark.parametrize("prec,tol,bound", [(PREC_F64, 1e-13, 1e-12), (PREC_F32, 1e-11, 1e-10)])
def test_batch_matches_oracle_and_individual(prec, tol, bound):
    lats, xs = [], []
    for i, dims in enumerate(SHAPES):
        u, src = _inputs(i, dims)
        lat = Lattice(dims)
        lat.build_links(torch.from_numpy(u).cuda(), 1.0)
        lats.append(lat)
        xs.append(torch.from_numpy(src).cuda())
    ys, stats = overlap_apply_batch(lats, xs, n=ORDER, tol=tol, prec=prec)
    for i, (lat, x, y) in enumerate(zip(lats, xs, ys)):
        assert relerr(y.cpu().numpy(), _oracle(i)) < bound, i
        y1, _ = lat.overlap_apply(x, n=ORDER, tol=tol, prec=prec)
        assert relerr(y.cpu().numpy(), y1.cpu().numpy()) < bound, i
