"""Batched overlap application over independent lattices of uneven volume
(concurrent streams, graph-replayed solver iterations, autotuned stencil):
identical results to per-lattice calls and to the oracle."""
import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, overlap
from paper_1701_00726_gb300 import PREC_F32, PREC_F64, Lattice, overlap_apply_batch

pytestmark = pytest.mark.gpu


def relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


@pytest.mark.parametrize("prec,tol,bound", [(PREC_F64, 1e-12, 1e-10), (PREC_F32, 1e-10, 1e-8)])
def test_batch_matches_individual_and_oracle(prec, tol, bound):
    shapes = [(4, 4, 4, 4), (6, 4, 4, 2), (4, 4, 2, 6), (2, 2, 2, 8)]
    lats, xs, us = [], [], []
    for i, dims in enumerate(shapes):
        u = sf.gauge_field(dims, 20 + i, 0.1, 3)
        lat = Lattice(dims)
        lat.build_links(torch.from_numpy(u).cuda(), 1.0)
        lats.append(lat)
        us.append(u)
        nr = 12 if i == 0 else 1
        src = sf.point_sources(dims) if i == 0 else sf.gaussian_source(dims, 1, 40 + i)
        xs.append(torch.from_numpy(src).cuda())
    ys, stats = overlap_apply_batch(lats, xs, n=12, tol=tol, prec=prec)
    for lat, x, y, u in zip(lats, xs, ys, us):
        y1, _ = lat.overlap_apply(x, n=12, tol=tol, prec=prec)
        assert relerr(y.cpu().numpy(), y1.cpu().numpy()) < bound
    # one lattice against the oracle
    want, _ = overlap.overlap_apply(dirac.DiracOperator(us[1], "bri", m0=-1.0, c_sw=1.0), xs[1].cpu().numpy(),
                                    1.0, 12, 1e-13)
    assert relerr(ys[1].cpu().numpy(), want) < bound
