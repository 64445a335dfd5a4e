"""Massive overlap solve with cascaded preconditioning (Secs. 4.2-4.4, Sec. 8)
on the GPU, verified with the oracle's forward operator: (D_ov + mt) x = bt
for the complete (Eq. upshot_complete) and traditional (Eq. upshot_traditional)
right-hand sides."""
import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, overlap
from paper_1701_00726_gb300 import PREC_F32, PREC_F64, Lattice

pytestmark = pytest.mark.gpu

RHO = 1.0


@pytest.mark.parametrize("complete,am,n_inner,prec", [(True, 0.1, 2, PREC_F64), (False, 0.5, 0, PREC_F64),
                                                      (True, 0.05, 2, PREC_F32)])
def test_massive_solve_residual_with_oracle(complete, am, n_inner, prec):
    dims = (4, 4, 3, 2)
    n_outer = 6
    u = sf.gauge_field(dims, 1, 0.1, 3)
    b = sf.gaussian_source(dims, 1, 1001)
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    x, st = lat.overlap_solve(torch.from_numpy(b).cuda(), n_outer, n_inner, rho=RHO, am=am, complete=complete,
                              tol=1e-10, prec=prec)
    assert st["converged"], st
    x = x.cpu().numpy()
    kern = dirac.DiracOperator(u, "bri", m0=-RHO, c_sw=1.0)
    dov_b, _ = overlap.overlap_apply(kern, b, RHO, n_outer, 1e-13)
    if complete:
        mt, bt = overlap.complete_mass_rhs(dov_b, b, RHO, am)
    else:
        mt, bt = overlap.traditional_mass_rhs(b, RHO, am)
    dov_x, _ = overlap.overlap_apply(kern, x, RHO, n_outer, 1e-13)
    res = np.linalg.norm((dov_x + mt * x - bt).ravel()) / np.linalg.norm(bt.ravel())
    assert res < 1e-9


def test_cascade_reduces_outer_iterations():
    dims = (4, 4, 4, 4)
    u = sf.gauge_field(dims, 1, 0.1, 3)
    b = torch.from_numpy(sf.gaussian_source(dims, 1, 1001)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    x0, s0 = lat.overlap_solve(b, 8, 0, am=0.05, tol=1e-9)
    x1, s1 = lat.overlap_solve(b, 8, 2, am=0.05, tol=1e-9)
    assert s0["converged"] and s1["converged"]
    assert s1["iterations"] < s0["iterations"]
    d = (x1 - x0).abs().max().item() / x0.abs().max().item()
    assert d < 1e-7
