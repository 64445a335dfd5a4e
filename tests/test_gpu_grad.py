"""Adjoint of the overlap application on the GPU (through the C ABI):
against the oracle gradient, against finite differences of the GPU forward
(8^4, FP64, KL order 12, 32 random link and source directions), and through
torch.autograd."""
import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import grad as ograd
from paper_1701_00726_gb300 import PREC_F32, PREC_F64, Lattice, overlap

pytestmark = pytest.mark.gpu


def relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _traceless_hermitian(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a + np.swapaxes(a, -1, -2).conj())
    return h - np.trace(h, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3


@pytest.mark.parametrize("am,anti", [(0.0, False), (0.3, True)])
def test_grad_vs_oracle(am, anti):
    """Ragged 6x5x4x3 lattice (every extent >= 3, so +d and -d hops land on different sites)."""
    dims = (6, 5, 4, 3)
    n = 6
    u = sf.gauge_field(dims, 91)
    eta = sf.gaussian_source(dims, 2, 92, normalize=True)
    psi = sf.gaussian_source(dims, 2, 93, normalize=True)
    lat = Lattice(dims, antiperiodic_t=anti)
    lat.build_links(torch.from_numpy(u).cuda(), 0.0)
    g_psi, g_u, st = lat.overlap_grad(torch.from_numpy(eta).cuda(), torch.from_numpy(psi).cuda(), n, am=am, tol=1e-13)
    assert st["converged"]
    w_psi, w_u = ograd.overlap_grad(u, eta, psi, 1.0, n, 1e-13, am=am, antiperiodic_t=anti)
    assert relerr(g_psi.cpu().numpy(), w_psi) < 1e-10
    assert relerr(g_u.cpu().numpy(), w_u) < 1e-10


@pytest.mark.parametrize("kernel,c_sw,am,anti", [("bri", 1.0, 0.1, False), ("wil", 1.0, 0.0, True),
                                                 ("wil", 0.0, 0.2, False)])
def test_grad_clover_and_wilson_vs_oracle(kernel, c_sw, am, anti):
    """Clover-term adjoint (Sec. 9 force ingredients) and the Wilson-kernel overlap's adjoint
    against the oracle gradient on the ragged 6x5x4x3 lattice, within 1e-10."""
    dims = (6, 5, 4, 3)
    n = 6
    u = sf.gauge_field(dims, 94)
    eta = sf.gaussian_source(dims, 2, 95, normalize=True)
    psi = sf.gaussian_source(dims, 2, 96, normalize=True)
    lat = Lattice(dims, antiperiodic_t=anti)
    lat.build_links(torch.from_numpy(u).cuda(), c_sw)
    lat.set_kernel(kernel)
    g_psi, g_u, st = lat.overlap_grad(torch.from_numpy(eta).cuda(), torch.from_numpy(psi).cuda(), n, am=am, tol=1e-13)
    assert st["converged"]
    w_psi, w_u = ograd.overlap_grad(u, eta, psi, 1.0, n, 1e-13, am=am, antiperiodic_t=anti, c_sw=c_sw, kernel=kernel)
    assert relerr(g_psi.cpu().numpy(), w_psi) < 1e-10
    assert relerr(g_u.cpu().numpy(), w_u) < 1e-10


def test_grad_finite_differences_8x4():
    """C5 workload: 8^4, FP64, KL order 12, unit-norm eta and psi; 32 random directions."""
    dims = (8, 8, 8, 8)
    n = 12
    u = sf.gauge_field(dims, 3)
    eta = torch.from_numpy(sf.gaussian_source(dims, 1, 1003, normalize=True)).cuda()
    psi = torch.from_numpy(sf.gaussian_source(dims, 1, 2003, normalize=True)).cuda()
    lat = Lattice(dims)
    ut = torch.from_numpy(u).cuda()
    lat.build_links(ut, 0.0)
    g_psi, g_u, st = lat.overlap_grad(eta, psi, n, tol=1e-14)
    gu = g_u.cpu().numpy()

    def loss(links, src):
        lat.build_links(links, 0.0)
        y, _ = lat.overlap_apply(src, n, tol=1e-14)
        return float(torch.vdot(eta.flatten(), y.flatten()).real)

    h = 1e-6
    worst = 0.0
    for k in range(32):
        if k % 2 == 0:  # link direction U -> exp(i h X) U
            x = _traceless_hermitian(u.shape[:5], 500 + k)
            up = torch.from_numpy(sf.su3_exp_i(h * x) @ u).cuda()
            um = torch.from_numpy(sf.su3_exp_i(-h * x) @ u).cuda()
            fd = (loss(up, psi) - loss(um, psi)) / (2 * h)
            an = float(np.einsum("...ba,...bc->...ac", gu.conj(), 1j * x @ u).trace(axis1=-2, axis2=-1).real.sum())
        else:  # source direction
            d = torch.from_numpy(sf.gaussian_source(dims, 1, 700 + k)).cuda()
            fd = (loss(ut, psi + h * d) - loss(ut, psi - h * d)) / (2 * h)
            an = float(torch.vdot(g_psi.flatten(), d.flatten()).real)
        worst = max(worst, abs(fd - an) / max(1.0, abs(fd)))
    assert worst < 1e-8


def test_autograd_function():
    dims = (4, 4, 4, 4)
    n = 4
    u = torch.from_numpy(sf.gauge_field(dims, 5)).cuda().requires_grad_(True)
    psi = torch.from_numpy(sf.gaussian_source(dims, 1, 6, normalize=True)).cuda().requires_grad_(True)
    eta = torch.from_numpy(sf.gaussian_source(dims, 1, 7, normalize=True)).cuda()
    lat = Lattice(dims)
    y = overlap(psi, u, lat, n, tol=1e-13)
    torch.vdot(eta.flatten(), y.flatten()).real.backward()
    g_psi, g_u, _ = lat.overlap_grad(eta, psi.detach(), n, tol=1e-13)
    assert relerr(psi.grad.cpu().numpy(), g_psi.cpu().numpy()) < 1e-12
    assert relerr(u.grad.cpu().numpy(), g_u.cpu().numpy()) < 1e-12


def test_grad_mixed_precision_matches_fp64():
    dims = (8, 8, 8, 8)
    u = sf.gauge_field(dims, 3)
    eta = torch.from_numpy(sf.gaussian_source(dims, 1, 11, normalize=True)).cuda()
    psi = torch.from_numpy(sf.gaussian_source(dims, 1, 12, normalize=True)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 0.0)
    g1, u1, _ = lat.overlap_grad(eta, psi, 12, tol=1e-12, prec=PREC_F64)
    g2, u2, st = lat.overlap_grad(eta, psi, 12, tol=1e-10, prec=PREC_F32)
    assert st["converged"]
    assert relerr(g2.cpu().numpy(), g1.cpu().numpy()) < 1e-8
    assert relerr(u2.cpu().numpy(), u1.cpu().numpy()) < 1e-8
