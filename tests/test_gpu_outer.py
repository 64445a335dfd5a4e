"""Massive overlap solve with cascaded preconditioning (Secs. 4.2-4.4, Sec. 8)
on the GPU, verified with the oracle's forward operator: the true residual
||(D_ov + mt) x - bt|| / ||bt|| of the GPU solution x, with D_ov applied by
the FP64 oracle, for the complete (Eq. upshot_complete) and traditional
(Eq. upshot_traditional) right-hand sides.

The shape is that of the FP64 16^3x32 workload (outer Kenney-Laub order 16,
cascade by order 4, am in {0.01, 0.1, 0.5}, c_SW = 1, stout-smeared field) on
a 4x4x3x3 lattice, small enough for the oracle, with every extent >= 3 so that
no hop wraps onto its own opposite.  The GPU solves to 5e-11 and the oracle's
residual must be below 1e-10; the oracle applies D_ov with its multi-shift
solve at 1e-13.
"""
import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, overlap
from paper_1701_00726_gb300 import PREC_F32, PREC_F64, Lattice

pytestmark = pytest.mark.gpu

RHO = 1.0
DIMS = (4, 4, 3, 3)
N_OUTER, N_INNER = 16, 4
GPU_TOL, BOUND = 5e-11, 1e-10


def _oracle_residual(u, kind, b, x, am, complete, n_outer):
    kern = dirac.DiracOperator(u, kind, m0=-RHO, c_sw=1.0)
    if complete:
        dov_b, _ = overlap.overlap_apply(kern, b, RHO, n_outer, 1e-13)
        mt, bt = overlap.complete_mass_rhs(dov_b, b, RHO, am)
    else:
        mt, bt = overlap.traditional_mass_rhs(b, RHO, am)
    dov_x, _ = overlap.overlap_apply(kern, x, RHO, n_outer, 1e-13)
    return np.linalg.norm((dov_x + mt * x - bt).ravel()) / np.linalg.norm(bt.ravel())


@pytest.mark.parametrize("am", [0.01, 0.1, 0.5])
@pytest.mark.parametrize("complete", [True, False])
def test_cascaded_solve_c2_shape(am, complete):
    u = sf.gauge_field(DIMS, 1, 0.1, 3)
    b = sf.gaussian_source(DIMS, 1, 1001)
    lat = Lattice(DIMS)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    x, st = lat.overlap_solve(torch.from_numpy(b).cuda(), N_OUTER, N_INNER, rho=RHO, am=am, complete=complete,
                              tol=GPU_TOL, prec=PREC_F64)
    assert st["converged"], st
    assert st["max_true_residual"] <= GPU_TOL
    assert _oracle_residual(u, "bri", b, x.cpu().numpy(), am, complete, N_OUTER) < BOUND


def test_cascaded_solve_mixed_precision():
    """The same solve with the FP32 inner multi-shift solves (FP64 refinement of every shift)."""
    am = 0.1
    u = sf.gauge_field(DIMS, 1, 0.1, 3)
    b = sf.gaussian_source(DIMS, 1, 1001)
    lat = Lattice(DIMS)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    x, st = lat.overlap_solve(torch.from_numpy(b).cuda(), N_OUTER, N_INNER, rho=RHO, am=am, complete=True,
                              tol=GPU_TOL, prec=PREC_F32)
    assert st["converged"], st
    assert _oracle_residual(u, "bri", b, x.cpu().numpy(), am, True, N_OUTER) < BOUND


@pytest.mark.parametrize("am", [0.01, 0.5])
def test_cascaded_solve_wilson_kernel(am):
    """Overlap with the Wilson kernel (Eq. def_wils inside Eq. def_over), same cascade."""
    u = sf.gauge_field(DIMS, 1, 0.1, 3)
    b = sf.gaussian_source(DIMS, 1, 1001)
    lat = Lattice(DIMS)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    lat.set_kernel("wil")
    x, st = lat.overlap_solve(torch.from_numpy(b).cuda(), N_OUTER, N_INNER, rho=RHO, am=am, complete=True,
                              tol=GPU_TOL, prec=PREC_F64)
    assert st["converged"], st
    assert _oracle_residual(u, "wil", b, x.cpu().numpy(), am, True, N_OUTER) < BOUND


def test_cascade_reduces_outer_iterations():
    """Sec. 8, Tab. 8: the cascade cuts the number of outer iterations; both solutions agree."""
    dims = (4, 4, 4, 4)
    u = sf.gauge_field(dims, 1, 0.1, 3)
    b = torch.from_numpy(sf.gaussian_source(dims, 1, 1001)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    x0, s0 = lat.overlap_solve(b, N_OUTER, 0, am=0.05, tol=1e-10)
    x1, s1 = lat.overlap_solve(b, N_OUTER, N_INNER, am=0.05, tol=1e-10)
    assert s0["converged"] and s1["converged"]
    assert s1["iterations"] < s0["iterations"]
    d = (x1 - x0).abs().max().item() / x0.abs().max().item()
    assert d < 1e-8
