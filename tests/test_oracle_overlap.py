"""Pins of the oracle's multi-shift CG and overlap operator.

* every shifted solution against a dense direct solve (2^4);
* the free-field overlap against the momentum-space closed form of App. A with
  the Kenney-Laub rational in place of [.]^{-1/2};
* the Krylov overlap against rho (1 + gamma5 f(H)) from a dense
  eigendecomposition of H (2^4 and, for the 4^4 / 12-source workload, 3072^2);
* exact algebraic identities: the Ginsparg-Wilson defect of the rational,
  D gamma5 + gamma5 D - D gamma5 D / rho = rho gamma5 (1 - f(H)^2), exact GW and
  sign^2 = 1 for the exact sign (Eqs. ginswils_one/two), and the contact term
  S_com - S_tra = I/(2 rho) (Eq. contact).
"""
import itertools

import numpy as np
import pytest

import synthetic_fields as sf
from oracle import dense, dirac, freefield, kl, mscg, overlap

RHO = 1.0


def _kernel(dims, seed, c_sw=0.0, eps=None, kind="bri"):
    u = sf.gauge_field(dims, seed, eps=eps)
    return dirac.DiracOperator(u, kind, m0=-RHO, c_sw=c_sw)


def test_multishift_vs_dense_solve():
    dims = (2, 2, 2, 2)
    op = _kernel(dims, 1, c_sw=1.0)
    b = sf.gaussian_source(dims, 1, 1001)
    _, _, sig = kl.kl_coeffs(6)
    xs, it = mscg.multishift_cg(op.normal, b, sig, 1e-12)
    a = dense.dense_matrix(op.normal, sf.lattice_shape(dims))
    for s, x in zip(sig, xs):
        want = np.linalg.solve(a + s * np.eye(a.shape[0]), b.ravel())
        np.testing.assert_allclose(x.ravel(), want, rtol=0, atol=1e-10 * np.abs(want).max())
    res = mscg.true_residuals(op.normal, b, sig, xs)
    assert max(res) < 1e-11
    assert 0 < it < 500


def test_free_field_overlap_closed_form():
    dims = (4, 2, 2, 2)
    op = _kernel(dims, 0, eps=0.0)
    n = 8
    r_of_y = lambda y: kl.rational_r(y, n)
    rng = np.random.default_rng(2)
    for k in [(0, 0, 0, 0), (1, 0, 1, 1), (3, 1, 0, 1), (2, 1, 1, 0)]:
        p = [2 * np.pi * k[m] / dims[m] for m in range(4)]
        xi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        lt, lz, ly, lx = sf.lattice_shape(dims)
        t, z, y, x = np.meshgrid(*[np.arange(v) for v in (lt, lz, ly, lx)], indexing="ij")
        ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[None, ..., None, None]
        src = ph * xi
        got, _ = overlap.overlap_apply(op, src, RHO, n, 1e-13)
        want = ph * (freefield.overlap_symbol(p, "bri", RHO, r_of_y) @ xi)
        np.testing.assert_allclose(got, want, atol=1e-10)


def _dense_overlap(op, nsite, n):
    d = dense.dense_matrix(op.apply, op.w.shape[1:5])
    g5 = dense.gamma5_dense(nsite)
    h = g5 @ d
    fh, lam = dense.hermitian_function(h, lambda v: kl.rational_pf(v, n))
    return d, g5, h, fh, lam


def test_overlap_vs_dense_eig_2x4():
    dims = (2, 2, 2, 2)
    n = 8
    op = _kernel(dims, 4, c_sw=1.0)
    d, g5, h, fh, lam = _dense_overlap(op, 16, n)
    b = sf.gaussian_source(dims, 3, 1004)
    got, info = overlap.overlap_apply(op, b, RHO, n, 1e-12)
    dov = RHO * (np.eye(d.shape[0]) + g5 @ fh)
    for r in range(3):
        want = dov @ b[r].ravel()
        np.testing.assert_allclose(got[r].ravel(), want, atol=1e-10 * np.abs(want).max())
        assert max(info[r]["residuals"]) < 1e-11
    # Massive traditional form (Eq. def_mass_traditional)
    am = 0.1
    gotm, _ = overlap.overlap_apply(op, b[:1], RHO, n, 1e-12, am=am)
    wantm = ((1 - am / (2 * RHO)) * dov + am * np.eye(d.shape[0])) @ b[0].ravel()
    np.testing.assert_allclose(gotm[0].ravel(), wantm, atol=1e-10 * np.abs(wantm).max())


def test_ginsparg_wilson_identities_dense():
    dims = (2, 2, 2, 2)
    n = 4
    op = _kernel(dims, 5)
    d, g5, h, fh, lam = _dense_overlap(op, 16, n)
    eye = np.eye(d.shape[0])
    dov = RHO * (eye + g5 @ fh)
    gw = dov @ g5 + g5 @ dov - dov @ g5 @ dov / RHO
    np.testing.assert_allclose(gw, RHO * g5 @ (eye - fh @ fh), atol=1e-12)
    # normality defect D D^dag - D^dag D = rho^2 (gamma5 f^2 gamma5 - f^2)
    np.testing.assert_allclose(dov @ dov.conj().T - dov.conj().T @ dov,
                               RHO ** 2 * (g5 @ fh @ fh @ g5 - fh @ fh), atol=1e-12)
    # exact sign: sign^2 = 1 and exact GW (Eqs. ginswils_one, ginswils_two)
    sgn, _ = dense.hermitian_function(h, np.sign)
    np.testing.assert_allclose(sgn @ sgn, eye, atol=1e-12)
    dex = RHO * (eye + g5 @ sgn)
    np.testing.assert_allclose(dex @ g5 + g5 @ dex, dex @ g5 @ dex / RHO, atol=1e-12)
    np.testing.assert_allclose(dex.conj().T + dex, dex.conj().T @ dex / RHO, atol=1e-12)
    # the rational is within max |1 - f(lambda)^2| of GW
    defect = np.linalg.norm(gw, 2)
    assert defect <= RHO * np.max(np.abs(1 - kl.rational_pf(lam, n) ** 2)) + 1e-12


def test_complete_vs_traditional_contact_term():
    """Eq. contact: S_com - S_tra = I / (2 rho), with D_ov from the rational."""
    dims = (2, 2, 2, 2)
    op = _kernel(dims, 6)
    d, g5, h, fh, lam = _dense_overlap(op, 16, 6)
    eye = np.eye(d.shape[0])
    dov = RHO * (eye + g5 @ fh)
    am = 0.3
    b = sf.gaussian_source(dims, 1, 1006)[0].ravel()
    mt_t, bt_t = overlap.traditional_mass_rhs(b, RHO, am)
    mt_c, bt_c = overlap.complete_mass_rhs(dov @ b, b, RHO, am)
    assert mt_t == pytest.approx(mt_c)
    x_t = np.linalg.solve(dov + mt_t * eye, bt_t)   # D_m^tra x = b (Eq. upshot_traditional)
    x_c = np.linalg.solve(dov + mt_c * eye, bt_c)   # D_m^com x = b (Eq. upshot_complete)
    s_tra_b = x_t - dov @ x_t / (2 * RHO)           # (1 - D/(2 rho)) attached, Eq. inv_traditional
    np.testing.assert_allclose(x_c - s_tra_b, b / (2 * RHO), atol=1e-11)


@pytest.mark.slow
def test_c1_workload_4x4_dense():
    """4^4, c_SW = 0, KL order 8, 12 Gaussian sources, tol 1e-12, vs dense f(H) (3072^2)."""
    dims = (4, 4, 4, 4)
    n = 8
    op = _kernel(dims, 0)
    d, g5, h, fh, lam = _dense_overlap(op, 256, n)
    b = sf.gaussian_source(dims, 12, 1000)
    got, info = overlap.overlap_apply(op, b, RHO, n, 1e-12)
    dov = RHO * (np.eye(d.shape[0]) + g5 @ fh)
    want = (dov @ b.reshape(12, -1).T).T
    err = np.abs(got.reshape(12, -1) - want).max() / np.abs(want).max()
    assert err < 1e-10
    assert max(max(i["residuals"]) for i in info) < 1e-11
