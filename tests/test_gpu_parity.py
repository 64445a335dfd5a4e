"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several 128-site thread blocks with a ragged tail; the smallest
lattice 2^4 makes every neighbour wrap.  Tolerances: FP64 1e-12 relative
(max-norm), a single FP32 matvec 1e-5, BF16-stored links 1e-2 (8-bit
mantissa: each link element carries a relative rounding error up to 2^-9,
and the 80 hop terms add with random signs), solver results 1e-10.
"""
import functools

import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, kl, links, overlap
from paper_1701_00726_gb300 import PREC_F32, PREC_F32_BF16, PREC_F64, BriError, Lattice, kl_coeffs

pytestmark = pytest.mark.gpu

RAGGED = (6, 5, 4, 3)  # 360 sites: two full 128-site blocks and a ragged tail


def relerr(got, want):
    return float(np.abs(got - want).max() / max(np.abs(want).max(), 1e-300))


def _lattice(dims, u, c_sw=0.0, anti=False):
    lat = Lattice(dims, antiperiodic_t=anti)
    lat.build_links(torch.from_numpy(u).cuda().contiguous(), c_sw)
    return lat


def test_kl_coeffs_abi():
    for kind in (0, 1):
        for n in (1, 2, 5, 8, 12, 16, 32):
            for s in (1.0, 2.5):
                c0, w, sig = kl_coeffs(n, kind, s)
                oc0, ow, osig = kl.kl_coeffs(n, kind, s)
                assert abs(c0 - oc0) <= 1e-15 * max(1.0, abs(oc0))
                np.testing.assert_allclose(w, ow, rtol=2e-15)
                np.testing.assert_allclose(sig, osig, rtol=2e-15)
    with pytest.raises(BriError):
        kl_coeffs(0)
    with pytest.raises(BriError):
        kl_coeffs(33)


@pytest.mark.parametrize("anti", [False, True])
def test_links_vs_path_enumeration(anti):
    dims = (3, 4, 2, 3)
    u = sf.gauge_field(dims, 7)
    lat = _lattice(dims, u, anti=anti)
    got = lat.links().cpu().numpy()
    want = links.stored_links(links.offaxis_links(u, anti))
    assert np.abs(got - want).max() < 1e-13


@pytest.mark.parametrize("dims", [RAGGED, (2, 2, 2, 2)])
@pytest.mark.parametrize("c_sw", [0.0, 1.0])
@pytest.mark.parametrize("dagger", [False, True])
def test_bri_apply_f64(dims, c_sw, dagger):
    u = sf.gauge_field(dims, 3)
    x = sf.gaussian_source(dims, 3, 1003)
    m0 = -1.0
    lat = _lattice(dims, u, c_sw)
    y = lat.bri_apply(torch.from_numpy(x).cuda(), m0, dagger=dagger).cpu().numpy()
    op = dirac.DiracOperator(u, "bri", m0=m0, c_sw=c_sw)
    want = op.apply_dagger(x) if dagger else op.apply(x)
    assert relerr(y, want) < 1e-12


@pytest.mark.parametrize("dims", [RAGGED, (4, 4, 4, 4)])
@pytest.mark.parametrize("c_sw", [0.0, 1.0])
@pytest.mark.parametrize("dagger", [False, True])
def test_bri_apply_double_word(dims, c_sw, dagger):
    """The double-word FP32 operator (error-free transformations on the FP32 pipe) against the FP64
    oracle: FP64-class accuracy, 1e-13 of the largest output element; a zero source stays zero."""
    u = sf.gauge_field(dims, 11, 0.1, 3)
    x = sf.gaussian_source(dims, 3, 1011)
    x[1] = 0.0
    lat = _lattice(dims, u, c_sw)
    y = lat.bri_apply(torch.from_numpy(x).cuda(), -1.0, dagger=dagger, double_word=True).cpu().numpy()
    op = dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=c_sw)
    want = op.apply_dagger(x) if dagger else op.apply(x)
    assert relerr(y, want) < 1e-13
    assert np.abs(y[1]).max() == 0.0


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("dagger", [False, True])
def test_bri_apply_f32(bf16, dagger):
    dims = RAGGED
    u = sf.gauge_field(dims, 4)
    x = sf.gaussian_source(dims, 2, 1004)
    lat = _lattice(dims, u, 1.0)
    y = lat.bri_apply(torch.from_numpy(x).to(torch.complex64).cuda(), -1.0, dagger=dagger,
                      bf16_links=bf16).cpu().numpy()
    op = dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0)
    want = op.apply_dagger(x) if dagger else op.apply(x)
    assert relerr(y, want) < (1e-2 if bf16 else 1e-5)


@pytest.mark.parametrize("c_sw", [0.0, 1.0])
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("anti", [False, True])
def test_wils_apply(c_sw, dagger, anti):
    dims = RAGGED
    u = sf.gauge_field(dims, 5)
    x = sf.gaussian_source(dims, 2, 1005)
    lat = _lattice(dims, u, c_sw, anti)
    op = dirac.DiracOperator(u, "wil", m0=-0.7, c_sw=c_sw, antiperiodic_t=anti)
    want = op.apply_dagger(x) if dagger else op.apply(x)
    y64 = lat.wils_apply(torch.from_numpy(x).cuda(), -0.7, dagger=dagger).cpu().numpy()
    assert relerr(y64, want) < 1e-12
    y32 = lat.wils_apply(torch.from_numpy(x).to(torch.complex64).cuda(), -0.7, dagger=dagger).cpu().numpy()
    assert relerr(y32, want) < 1e-5


def test_antiperiodic_bri():
    dims = RAGGED
    u = sf.gauge_field(dims, 6)
    x = sf.gaussian_source(dims, 1, 1006)
    lat = _lattice(dims, u, 1.0, anti=True)
    y = lat.bri_apply(torch.from_numpy(x).cuda(), -1.0).cpu().numpy()
    want = dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0, antiperiodic_t=True).apply(x)
    assert relerr(y, want) < 1e-12


def test_invalid_arguments():
    dims = (4, 4, 4, 4)
    u = sf.gauge_field(dims, 0)
    lat = Lattice(dims)
    x = torch.zeros((1,) + sf.lattice_shape(dims) + (4, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(BriError):  # links not built yet
        lat.bri_apply(x, -1.0)
    lat.build_links(torch.from_numpy(u).cuda(), 0.0)
    with pytest.raises(BriError):  # wrong size
        lat.bri_apply(x[..., :2], -1.0)
    with pytest.raises(BriError):
        lat.overlap_apply(x, n=0)
    with pytest.raises(BriError):
        lat.overlap_apply(x, n=8, rho=2.5)
    with pytest.raises(BriError):
        Lattice((1, 4, 4, 4))


@pytest.mark.parametrize("prec,tol,bound", [(PREC_F64, 1e-13, 1e-12), (PREC_F32, 1e-11, 1e-10),
                                            (PREC_F32_BF16, 1e-11, 1e-10)])
def test_overlap_c1_workload(prec, tol, bound):
    """4^4, c_SW = 0, rho = 1, KL order 8, 12 Gaussian sources (FP64, mixed FP32, mixed BF16 links)."""
    dims = (4, 4, 4, 4)
    u = sf.gauge_field(dims, 0)
    x = sf.gaussian_source(dims, 12, 1000)
    lat = _lattice(dims, u)
    y, st = lat.overlap_apply(torch.from_numpy(x).cuda(), n=8, rho=1.0, tol=tol, prec=prec, want_true_residual=True)
    assert st["converged"]
    assert st["max_true_residual"] < 10 * tol
    want, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0), x, 1.0, 8, 1e-13)
    assert relerr(y.cpu().numpy(), want) < bound


def test_overlap_clover_massive_and_sign():
    dims = RAGGED
    u = sf.gauge_field(dims, 8)
    x = sf.gaussian_source(dims, 2, 1008)
    lat = _lattice(dims, u, 1.0)
    kern = dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0)
    xt = torch.from_numpy(x).cuda()
    y, st = lat.overlap_apply(xt, n=6, rho=1.0, am=0.1, tol=1e-13)
    want, _ = overlap.overlap_apply(kern, x, 1.0, 6, 1e-13, am=0.1)
    assert relerr(y.cpu().numpy(), want) < 1e-12
    s, _ = lat.sign_apply(xt, n=6, rho=1.0, tol=1e-13)
    swant, _ = overlap.sign_apply(kern, x, 6, 1e-13)
    assert relerr(s.cpu().numpy(), swant) < 1e-12
    # upper-diagonal family g_{2n} (Tab. 6)
    s1, _ = lat.sign_apply(xt, n=3, rho=1.0, tol=1e-13, kind=1)
    swant1, _ = overlap.sign_apply(kern, x, 3, 1e-13, kind=1)
    assert relerr(s1.cpu().numpy(), swant1) < 1e-12


def test_bri_apply_full_size_sampled():
    """24^3 x 48 (the benchmark lattice), FP32 spinors / FP32 and BF16 links, 12 sources:
    sampled sites against the per-site oracle, and gamma5-hermiticity of the FP64 path."""
    dims = (24, 24, 24, 48)
    u = sf.gauge_field(dims, 1, 0.1, 3, device="cuda")
    x = sf.gaussian_source(dims, 12, 1001)
    lat = _lattice(dims, u, 1.0)
    xt = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(0)
    sites = [tuple(int(rng.integers(0, L)) for L in dims) for _ in range(12)]
    sites += [(0, 0, 0, 0), (23, 23, 23, 47), (0, 23, 0, 47)]
    want = dirac.apply_at_sites(u, "bri", -1.0, 1.0, x, sites)
    for bf16, bound in ((False, 1e-5), (True, 1e-2)):
        y = lat.bri_apply(xt.to(torch.complex64), -1.0, bf16_links=bf16)
        got = np.stack([y[:, st, sz, sy, sx].cpu().numpy() for (sx, sy, sz, st) in sites], axis=1)
        assert relerr(got, want) < bound
    y64 = lat.bri_apply(xt[:2], -1.0)
    got = np.stack([y64[:, st, sz, sy, sx].cpu().numpy() for (sx, sy, sz, st) in sites], axis=1)
    assert relerr(got, want[:2]) < 1e-12
    # <phi, D psi> = <D^dagger phi, psi>
    phi, psi = xt[0:1], xt[1:2]
    lhs = torch.vdot(phi.flatten(), lat.bri_apply(psi, -1.0).flatten())
    rhs = torch.vdot(lat.bri_apply(phi, -1.0, dagger=True).flatten(), psi.flatten())
    assert abs((lhs - rhs).item()) < 1e-11 * abs(lhs.item())


@pytest.mark.parametrize("prec", [PREC_F32, PREC_F32_BF16])
def test_mixed_order16_true_residuals(prec):
    """KL order 16 (smallest shift 2.3e-3), stout-smeared 8^4 field, c_SW = 1: every shift's FP64
    true residual reaches the requested 1e-10 (FP32 and BF16 links in the first phase)."""
    dims = (8, 8, 8, 8)
    u = sf.gauge_field(dims, 1, 0.1, 3)
    x = sf.gaussian_source(dims, 3, 1001)
    lat = _lattice(dims, u, 1.0)
    xt = torch.from_numpy(x).cuda()
    y, st = lat.overlap_apply(xt, n=16, rho=1.0, tol=1e-10, prec=prec, want_true_residual=True)
    assert st["converged"]
    assert st["max_true_residual"] <= 1e-10


@pytest.mark.parametrize("prec", [PREC_F32, PREC_F32_BF16])
def test_mixed_order16_vs_oracle(prec):
    """The benchmark's Kenney-Laub order 16 in mixed precision against the FP64 oracle on the
    ragged lattice (stout-smeared field, c_SW = 1): within 1e-10."""
    dims = RAGGED
    u = sf.gauge_field(dims, 1, 0.1, 3)
    x = sf.gaussian_source(dims, 1, 1011)
    lat = _lattice(dims, u, 1.0)
    y, st = lat.overlap_apply(torch.from_numpy(x).cuda(), n=16, rho=1.0, tol=1e-11, prec=prec)
    assert st["converged"]
    assert relerr(y.cpu().numpy(), _oracle_order16_ragged()) < 1e-10


@functools.lru_cache(maxsize=None)
def _oracle_order16_ragged():
    u = sf.gauge_field(RAGGED, 1, 0.1, 3)
    x = sf.gaussian_source(RAGGED, 1, 1011)
    want, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), x, 1.0, 16, 1e-13)
    return want


def test_mixed_many_rhs():
    """48 right-hand sides (more than the 32-system correction batches and the reduction grid's
    per-system split) on 8^4: mixed result against the FP64 path, every shift at the requested
    true residual."""
    dims = (8, 8, 8, 8)
    u = sf.gauge_field(dims, 2, 0.1, 3)
    x = torch.from_numpy(sf.gaussian_source(dims, 48, 1012)).cuda()
    lat = _lattice(dims, u, 1.0)
    y, st = lat.overlap_apply(x, n=4, rho=1.0, tol=1e-11, prec=PREC_F32, want_true_residual=True)
    assert st["converged"]
    assert st["max_true_residual"] <= 1e-11
    y64, _ = lat.overlap_apply(x, n=4, rho=1.0, tol=1e-13, prec=PREC_F64)
    assert relerr(y.cpu().numpy(), y64.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("prec,tol,bound", [(PREC_F64, 1e-13, 1e-12), (PREC_F32, 1e-11, 1e-10)])
def test_overlap_wilson_kernel(prec, tol, bound):
    """D_ov with the Wilson kernel (Eq. def_wils inside Eq. def_over), c_SW = 1, massive
    traditional form and the sign function of the upper-diagonal family, against the oracle."""
    dims = RAGGED
    u = sf.gauge_field(dims, 8, 0.1, 3)
    x = sf.gaussian_source(dims, 2, 1013)
    lat = _lattice(dims, u, 1.0)
    lat.set_kernel("wil")
    xt = torch.from_numpy(x).cuda()
    want, swant1 = _oracle_wilson_overlap()
    y, st = lat.overlap_apply(xt, n=8, rho=1.0, am=0.1, tol=tol, prec=prec)
    assert st["converged"]
    assert relerr(y.cpu().numpy(), want) < bound
    s1, _ = lat.sign_apply(xt, n=4, rho=1.0, tol=tol, prec=prec, kind=1)
    assert relerr(s1.cpu().numpy(), swant1) < bound
    lat.set_kernel("bri")
    yb, _ = lat.overlap_apply(xt, n=8, rho=1.0, am=0.1, tol=tol, prec=prec)
    assert relerr(yb.cpu().numpy(), want) > 1e-3  # the selector really switches the kernel


@functools.lru_cache(maxsize=None)
def _oracle_wilson_overlap():
    u = sf.gauge_field(RAGGED, 8, 0.1, 3)
    x = sf.gaussian_source(RAGGED, 2, 1013)
    kern = dirac.DiracOperator(u, "wil", m0=-1.0, c_sw=1.0)
    want, _ = overlap.overlap_apply(kern, x, 1.0, 8, 1e-13, am=0.1)
    swant1, _ = overlap.sign_apply(kern, x, 4, 1e-13, kind=1)
    return want, swant1


@pytest.mark.parametrize("force", ["0,128,1", "1,128,1", "0,64,1", "1,64,1", "2,128,1", "2,64,1", "3,128,1",
                                   "3,64,1", "0,128,2", "0,128,4"])
def test_bri_apply_every_launch_configuration(force, monkeypatch):
    """Every stencil launch configuration the autotuner can pick gives the oracle's result
    (5 right-hand sides: groups plus a remainder)."""
    monkeypatch.setenv("BRI_STENCIL_FORCE", force)
    dims = RAGGED
    u = sf.gauge_field(dims, 9)
    x = sf.gaussian_source(dims, 5, 1009)
    lat = _lattice(dims, u, 1.0)
    op = dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0)
    for dagger in (False, True):
        y = lat.bri_apply(torch.from_numpy(x).to(torch.complex64).cuda(), -1.0, dagger=dagger).cpu().numpy()
        want = op.apply_dagger(x) if dagger else op.apply(x)
        assert relerr(y, want) < 1e-5


@functools.lru_cache(maxsize=None)
def _oracle_sign_three_rhs():
    u = sf.gauge_field(RAGGED, 10, 0.1, 3)
    x = sf.gaussian_source(RAGGED, 3, 1019)
    want, _ = overlap.sign_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), x, 8, 1e-13)
    return u, x, want


@pytest.mark.parametrize("force", ["0,128,1", "1,128,1", "2,128,1", "2,64,1", "3,128,1", "3,64,1", "0,128,2"])
def test_mixed_solve_every_launch_configuration(force, monkeypatch):
    """The mixed-precision sign function with every stencil configuration forced (each D^dagger
    launch of the FP32 solve carries the fused shift and dot-product epilogue; 3 right-hand sides:
    a two-rhs group plus a remainder) matches the oracle within 1e-10."""
    monkeypatch.setenv("BRI_STENCIL_FORCE", force)
    u, x, want = _oracle_sign_three_rhs()
    lat = _lattice(RAGGED, u, 1.0)
    y, st = lat.sign_apply(torch.from_numpy(x).cuda(), n=8, rho=1.0, tol=1e-11, prec=PREC_F32)
    assert st["converged"]
    assert relerr(y.cpu().numpy(), want) < 1e-10


def test_zero_source_and_free_field():
    """Degenerate inputs: a zero source among non-zero ones gives exactly zero (the solver stops that
    system at its zero norm); on the free field (U = 1, where the clover term vanishes) the overlap
    equals the oracle, whose free-field form is pinned to App. A's momentum-space expression."""
    dims = RAGGED
    u = sf.gauge_field(dims, 0, eps=0.0)
    x = sf.gaussian_source(dims, 3, 1021)
    x[1] = 0.0
    lat = _lattice(dims, u, 1.0)
    y, st = lat.overlap_apply(torch.from_numpy(x).cuda(), n=8, rho=1.0, tol=1e-13)
    assert st["converged"]
    got = y.cpu().numpy()
    assert np.abs(got[1]).max() == 0.0
    want, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), x, 1.0, 8, 1e-13)
    assert relerr(got, want) < 1e-12


def test_full_size_overlap_properties():
    """The benchmark's workload size (24^3 x 48, stout-smeared field, c_SW = 1, KL order 16, mixed
    precision): every shift's FP64 true residual reaches 1e-10, and D_ov is gamma5-hermitian,
    <phi, D psi> = <gamma5 D gamma5 phi, psi>, to the accuracy of the solves."""
    dims = (24, 24, 24, 48)
    u = sf.gauge_field(dims, 1, 0.1, 3, device="cuda")
    lat = _lattice(dims, u, 1.0)
    phi = torch.from_numpy(sf.gaussian_source(dims, 1, 1031, normalize=True)).cuda()
    psi = torch.from_numpy(sf.gaussian_source(dims, 1, 1032, normalize=True)).cuda()
    g5 = torch.tensor([1.0, 1.0, -1.0, -1.0], dtype=torch.complex128, device="cuda").view(4, 1)
    d_psi, st = lat.overlap_apply(psi, n=16, rho=1.0, tol=1e-10, prec=PREC_F32, want_true_residual=True)
    assert st["converged"]
    assert st["max_true_residual"] <= 1e-10
    d_phi, _ = lat.overlap_apply((phi * g5).contiguous(), n=16, rho=1.0, tol=1e-10, prec=PREC_F32)
    lhs = torch.vdot(phi.flatten(), d_psi.flatten())
    rhs = torch.vdot((d_phi * g5).flatten(), psi.flatten())
    assert abs((lhs - rhs).item()) <= 1e-8 * max(abs(lhs.item()), 1.0)
