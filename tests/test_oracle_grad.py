"""Pin of the oracle gradient of L = Re<eta, D_m psi> against finite differences
of a dense evaluation of L (eigendecomposition of H on 2^4: no Krylov noise).
Link directions U -> exp(i h X) U, X traceless Hermitian per link, give
dL/dh = sum Re tr(G^dagger i X U)."""
import numpy as np
import pytest

import synthetic_fields as sf
from oracle import dense, dirac, grad, kl

RHO = 1.0


def dense_loss(u, eta, psi, n, am=0.0, anti=False):
    dims_shape = u.shape[:4]
    op = dirac.DiracOperator(u, "bri", m0=-RHO, antiperiodic_t=anti)
    d = dense.dense_matrix(op.apply, dims_shape)
    nsite = int(np.prod(dims_shape))
    g5 = dense.gamma5_dense(nsite)
    fh, _ = dense.hermitian_function(g5 @ d, lambda v: kl.rational_pf(v, n))
    dov = RHO * (np.eye(d.shape[0]) + g5 @ fh)
    dm = (1 - am / (2 * RHO)) * dov + am * np.eye(d.shape[0])
    return sum(float(np.vdot(eta[r].ravel(), dm @ psi[r].ravel()).real) for r in range(psi.shape[0]))


def traceless_hermitian(shape, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    h = 0.5 * (a + np.swapaxes(a, -1, -2).conj())
    return h - np.trace(h, axis1=-2, axis2=-1)[..., None, None] * np.eye(3) / 3


@pytest.mark.parametrize("am,anti", [(0.0, False), (0.2, True)])
def test_oracle_gradient_vs_dense_fd(am, anti):
    dims = (2, 2, 2, 2)
    n = 4
    u = sf.gauge_field(dims, 61)
    eta = sf.gaussian_source(dims, 2, 62, normalize=True)
    psi = sf.gaussian_source(dims, 2, 63, normalize=True)
    g_psi, gu = grad.overlap_grad(u, eta, psi, RHO, n, 1e-14, am=am, antiperiodic_t=anti)
    # links
    x = traceless_hermitian(u.shape[:5], 64)
    h = 1e-5
    up = sf.su3_exp_i(h * x) @ u
    um = sf.su3_exp_i(-h * x) @ u
    fd = (dense_loss(up, eta, psi, n, am, anti) - dense_loss(um, eta, psi, n, am, anti)) / (2 * h)
    an = float(np.sum(np.einsum("...ba,...bc->...ac", gu.conj(), 1j * x @ u).trace(axis1=-2, axis2=-1).real))
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd))
    # source direction (L is linear in psi)
    delta = sf.gaussian_source(dims, 2, 65)
    fdp = (dense_loss(u, eta, psi + 1e-3 * delta, n, am, anti)
           - dense_loss(u, eta, psi - 1e-3 * delta, n, am, anti)) / 2e-3
    assert abs(fdp - float(np.vdot(g_psi.ravel(), delta.ravel()).real)) <= 1e-9 * max(1.0, abs(fdp))


def test_oracle_gradient_single_link_directions():
    """Perturb one link at a time (all four directions at one site): catches a
    wrong path position or a misplaced dagger that a global direction could hide."""
    dims = (2, 2, 2, 2)
    n = 3
    u = sf.gauge_field(dims, 71)
    eta = sf.gaussian_source(dims, 1, 72, normalize=True)
    psi = sf.gaussian_source(dims, 1, 73, normalize=True)
    _, gu = grad.overlap_grad(u, eta, psi, RHO, n, 1e-14)
    h = 1e-5
    for (t, z, y, xx, mu, seed) in [(0, 0, 0, 0, 0, 1), (1, 0, 1, 0, 3, 2), (0, 1, 1, 1, 1, 3), (1, 1, 0, 1, 2, 4)]:
        x = traceless_hermitian((), 80 + seed)
        up, um = u.copy(), u.copy()
        up[t, z, y, xx, mu] = sf.su3_exp_i(h * x) @ u[t, z, y, xx, mu]
        um[t, z, y, xx, mu] = sf.su3_exp_i(-h * x) @ u[t, z, y, xx, mu]
        fd = (dense_loss(up, eta, psi, n) - dense_loss(um, eta, psi, n)) / (2 * h)
        an = float(np.trace(gu[t, z, y, xx, mu].conj().T @ (1j * x @ u[t, z, y, xx, mu])).real)
        assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd))


def _clover_loss(u, uvec, vvec, c_sw, anti):
    from oracle.links import apply_time_bc
    cl = dirac.clover_field(apply_time_bc(u, anti), c_sw)
    cv = np.einsum("...satb,r...tb->r...sa", cl, vvec)
    return float(np.vdot(uvec.ravel(), cv.ravel()).real)


@pytest.mark.parametrize("anti", [False, True])
def test_oracle_clover_gradient_vs_fd(anti):
    """Re<u, C v> alone (no solve) on a 3x4x3x3 lattice: every extent >= 3, so the
    four leaves of a plane use distinct links; one global and four single-link directions."""
    from oracle.links import apply_time_bc
    dims = (3, 4, 3, 3)
    c_sw = 1.3
    u = sf.gauge_field(dims, 66)
    uvec = sf.gaussian_source(dims, 1, 67)
    vvec = sf.gaussian_source(dims, 1, 68)
    gu = grad.clover_link_gradient(apply_time_bc(u, anti), c_sw, [(uvec, vvec, 1.0)])
    if anti:
        gu[-1, :, :, :, 3] *= -1.0
    h = 1e-5
    x = traceless_hermitian(u.shape[:5], 69)
    fd = (_clover_loss(sf.su3_exp_i(h * x) @ u, uvec, vvec, c_sw, anti)
          - _clover_loss(sf.su3_exp_i(-h * x) @ u, uvec, vvec, c_sw, anti)) / (2 * h)
    an = float(np.sum(np.einsum("...ba,...bc->...ac", gu.conj(), 1j * x @ u).trace(axis1=-2, axis2=-1).real))
    assert abs(fd - an) <= 1e-8 * max(1.0, abs(fd))
    for (t, z, y, xx, mu, seed) in [(0, 0, 0, 0, 0, 1), (2, 1, 3, 2, 3, 2), (1, 2, 0, 1, 1, 3), (2, 2, 2, 0, 2, 4)]:
        xs = traceless_hermitian((), 90 + seed)
        up, um = u.copy(), u.copy()
        up[t, z, y, xx, mu] = sf.su3_exp_i(h * xs) @ u[t, z, y, xx, mu]
        um[t, z, y, xx, mu] = sf.su3_exp_i(-h * xs) @ u[t, z, y, xx, mu]
        fd1 = (_clover_loss(up, uvec, vvec, c_sw, anti) - _clover_loss(um, uvec, vvec, c_sw, anti)) / (2 * h)
        an1 = float(np.trace(gu[t, z, y, xx, mu].conj().T @ (1j * xs @ u[t, z, y, xx, mu])).real)
        assert abs(fd1 - an1) <= 1e-8 * max(1.0, abs(fd1))


def dense_loss_k(u, eta, psi, n, kernel, c_sw, am=0.0, anti=False):
    op = dirac.DiracOperator(u, kernel, m0=-RHO, c_sw=c_sw, antiperiodic_t=anti)
    dims_shape = u.shape[:4]
    d = dense.dense_matrix(op.apply, dims_shape)
    nsite = int(np.prod(dims_shape))
    g5 = dense.gamma5_dense(nsite)
    fh, _ = dense.hermitian_function(g5 @ d, lambda v: kl.rational_pf(v, n))
    dov = RHO * (np.eye(d.shape[0]) + g5 @ fh)
    dm = (1 - am / (2 * RHO)) * dov + am * np.eye(d.shape[0])
    return sum(float(np.vdot(eta[r].ravel(), dm @ psi[r].ravel()).real) for r in range(psi.shape[0]))


@pytest.mark.parametrize("kernel,c_sw,am,anti", [("bri", 1.0, 0.1, False), ("wil", 0.0, 0.0, True),
                                                 ("wil", 1.0, 0.2, False)])
def test_oracle_gradient_clover_and_wilson_vs_dense_fd(kernel, c_sw, am, anti):
    """The overlap gradient with the clover term and with the Wilson kernel, against dense FD on 2^4."""
    dims = (2, 2, 2, 2)
    n = 4
    u = sf.gauge_field(dims, 161)
    eta = sf.gaussian_source(dims, 1, 162, normalize=True)
    psi = sf.gaussian_source(dims, 1, 163, normalize=True)
    g_psi, gu = grad.overlap_grad(u, eta, psi, RHO, n, 1e-14, am=am, antiperiodic_t=anti, c_sw=c_sw, kernel=kernel)
    x = traceless_hermitian(u.shape[:5], 164)
    h = 1e-5
    fd = (dense_loss_k(sf.su3_exp_i(h * x) @ u, eta, psi, n, kernel, c_sw, am, anti)
          - dense_loss_k(sf.su3_exp_i(-h * x) @ u, eta, psi, n, kernel, c_sw, am, anti)) / (2 * h)
    an = float(np.sum(np.einsum("...ba,...bc->...ac", gu.conj(), 1j * x @ u).trace(axis1=-2, axis2=-1).real))
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd))
    delta = sf.gaussian_source(dims, 1, 165)
    fdp = (dense_loss_k(u, eta, psi + 1e-3 * delta, n, kernel, c_sw, am, anti)
           - dense_loss_k(u, eta, psi - 1e-3 * delta, n, kernel, c_sw, am, anti)) / 2e-3
    assert abs(fdp - float(np.vdot(g_psi.ravel(), delta.ravel()).real)) <= 1e-9 * max(1.0, abs(fdp))
