"""Pins of the oracle's kernels (links, stencils, clover) against what the
paper and the mathematics fix: the momentum-space forms of App. A on plane
waves, gamma matrix algebra, the mirror identity of App. C, pure-gauge and
gauge-covariance identities, gamma5-hermiticity (Sec. 4) and a by-hand path
walk with explicit index arithmetic.
"""
import itertools

import numpy as np
import pytest

import synthetic_fields as sf
from oracle import conventions as cv
from oracle import dense, dirac, freefield, links

DIMS_RAGGED = (4, 2, 3, 2)


def _plane_wave(dims, p, xi):
    lt, lz, ly, lx = sf.lattice_shape(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return phase[None, ..., None, None] * xi[None, None, None, None, None]


def test_gamma_algebra():
    g, g5 = cv.gammas()
    for mu in range(4):
        np.testing.assert_allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            ac = g[mu] @ g[nu] + g[nu] @ g[mu]
            np.testing.assert_allclose(ac, 2 * np.eye(4) * (mu == nu), atol=1e-15)
    np.testing.assert_allclose(g5, np.diag([1, 1, -1, -1]), atol=1e-15)


def test_offset_numbering():
    offs = cv.all_offsets()
    assert offs[40] == (0, 0, 0, 0)
    for i, d in enumerate(offs):
        assert cv.nu_index(d) == i
        assert offs[80 - i] == tuple(-c for c in d)  # nu and 82 - nu opposite
    for d in cv.stored_offsets():
        ms = [c for c in reversed(d) if c != 0][0]
        assert ms == -1
    assert sum(1 for d in offs if cv.hops(d) > 0) == 80


@pytest.mark.parametrize("kind", ["bri", "wil"])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_plane_waves_free_field(kind, antiperiodic):
    """App. A: on U = 1, D e^{ipn} xi = e^{ipn} D(p) xi at every lattice momentum."""
    dims = DIMS_RAGGED
    u = sf.gauge_field(dims, 0, eps=0.0)
    m0 = -0.37
    op = dirac.DiracOperator(u, kind, m0=m0, antiperiodic_t=antiperiodic)
    rng = np.random.default_rng(5)
    for k in itertools.product(*[range(L) for L in dims]):
        p = [2 * np.pi * k[m] / dims[m] for m in range(4)]
        if antiperiodic:
            p[3] = (2 * k[3] + 1) * np.pi / dims[3]
        xi = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        x = _plane_wave(dims, p, xi)
        sym, _, _ = freefield.kernel_symbol(p, kind, m0)
        want = _plane_wave(dims, p, sym @ xi)
        np.testing.assert_allclose(op.apply(x), want, atol=1e-13)


def test_stencil_weight_sums():
    # Delta annihilates constants; nabla^iso weights are odd; 54 offsets carry nabla_mu (App. C)
    assert sum(dirac.lap_bri_weight(d) for d in cv.all_offsets()) == pytest.approx(0.0, abs=1e-15)
    for mu in range(4):
        nz = [d for d in cv.all_offsets() if dirac.nabla_iso_weight(d, mu) != 0.0]
        assert len(nz) == 54
    assert dirac.lap_bri_weight((0, 0, 0, 0)) == pytest.approx(-15 / 4)
    for d in cv.all_offsets():
        k = cv.hops(d)
        if k:
            assert dirac.lap_bri_weight(d) == pytest.approx(2.0 ** (4 - k) / 64)
            for mu in range(4):
                if d[mu]:
                    assert dirac.nabla_iso_weight(d, mu) == pytest.approx(d[mu] * 4.0 ** (4 - k) / 432)


def test_mirror_identity():
    """App. C: W_nu(n) = W_{82-nu}(n + nu)^dagger."""
    u = sf.gauge_field(DIMS_RAGGED, 3)
    w = links.offaxis_links(u)
    for i, d in enumerate(cv.all_offsets()):
        np.testing.assert_allclose(w[i], cv.dag(cv.shift_by(w[80 - i], d)), atol=1e-14)


def test_pure_gauge_links():
    """U_mu(n) = O(n) O(n+mu)^dag gives W_d(n) = O(n) O(n+d)^dag for every path average."""
    dims = (3, 2, 2, 4)
    shape = sf.lattice_shape(dims)
    om = sf.random_su3(shape, 11)
    u = np.stack([om @ cv.dag(cv.shift(om, mu, 1)) for mu in range(4)], axis=4)
    w = links.offaxis_links(u)
    for i, d in enumerate(cv.all_offsets()):
        np.testing.assert_allclose(w[i], om @ cv.dag(cv.shift_by(om, d)), atol=1e-13)


def test_links_by_hand_walk():
    """Explicit coordinate arithmetic for a few (site, offset) pairs."""
    dims = (3, 4, 2, 3)
    lx, ly, lz, lt = dims
    u = sf.gauge_field(dims, 7)
    w = links.offaxis_links(u)

    def link(pos, mu):
        x, y, z, t = pos
        return u[t % lt, z % lz, y % ly, x % lx, mu]

    for site, d in [((0, 0, 0, 0), (-1, 1, 0, -1)), ((2, 3, 1, 2), (1, 1, 1, 1)), ((1, 0, 1, 0), (0, -1, -1, 0))]:
        dims_nz = [m for m in range(4) if d[m]]
        acc = np.zeros((3, 3), dtype=complex)
        perms = list(itertools.permutations(dims_nz))
        for perm in perms:
            pos = list(site)
            prod = np.eye(3, dtype=complex)
            for mu in perm:
                if d[mu] > 0:
                    prod = prod @ link(pos, mu)
                    pos[mu] += 1
                else:
                    pos[mu] -= 1
                    prod = prod @ link(pos, mu).conj().T
            acc += prod
        acc /= len(perms)
        x, y, z, t = site
        np.testing.assert_allclose(w[cv.nu_index(d), t, z, y, x], acc, atol=1e-14)


@pytest.mark.parametrize("kind,c_sw", [("bri", 0.0), ("bri", 1.0), ("wil", 1.0)])
def test_gauge_covariance(kind, c_sw):
    dims = (2, 3, 2, 4)
    shape = sf.lattice_shape(dims)
    u = sf.gauge_field(dims, 21)
    om = sf.random_su3(shape, 22)
    ug = np.stack([om @ u[..., mu, :, :] @ cv.dag(cv.shift(om, mu, 1)) for mu in range(4)], axis=4)
    psi = sf.gaussian_source(dims, 2, 23)
    op = dirac.DiracOperator(u, kind, m0=-1.0, c_sw=c_sw)
    opg = dirac.DiracOperator(ug, kind, m0=-1.0, c_sw=c_sw)
    rot = lambda v: np.einsum("...ab,r...sb->r...sa", om, v)
    np.testing.assert_allclose(opg.apply(rot(psi)), rot(op.apply(psi)), atol=1e-12)


@pytest.mark.parametrize("kind,c_sw,anti", [("bri", 0.0, False), ("bri", 1.0, True), ("wil", 1.0, False)])
def test_gamma5_hermiticity_dense(kind, c_sw, anti):
    """gamma5 D gamma5 = D^dagger, checked on the dense matrix (Sec. 4)."""
    dims = (2, 2, 2, 2)
    u = sf.gauge_field(dims, 31)
    op = dirac.DiracOperator(u, kind, m0=-1.0, c_sw=c_sw, antiperiodic_t=anti)
    d = dense.dense_matrix(op.apply, sf.lattice_shape(dims))
    g5 = dense.gamma5_dense(16)
    np.testing.assert_allclose(g5 @ d @ g5, d.conj().T, atol=1e-13)


def test_clover_properties():
    dims = (2, 3, 2, 3)
    u = sf.gauge_field(dims, 41)
    c = dirac.clover_field(u, 1.0).reshape(sf.lattice_shape(dims) + (12, 12))
    np.testing.assert_allclose(c, np.swapaxes(c, -1, -2).conj(), atol=1e-14)  # Hermitian
    g5 = np.kron(np.diag([1, 1, -1, -1]), np.eye(3))
    np.testing.assert_allclose(g5 @ c, c @ g5, atol=1e-14)  # commutes with gamma5
    assert np.abs(c).max() > 0.05
    free = dirac.clover_field(sf.gauge_field(dims, 0, eps=0.0), 1.0)
    assert np.abs(free).max() < 1e-15
    np.testing.assert_allclose(np.trace(c, axis1=-2, axis2=-1), 0, atol=1e-13)


def test_clover_abelian_field_strength():
    """Commuting links U_mu = exp(i theta_mu T), T = diag(1,-1,0): every clover leaf is
    the counter-clockwise plaquette with corner n, n-mu, n-mu-nu or n-nu, so
    F_{mu nu}(n) = (1/4) sum_corners sin(phi_corner) T, phi the plaquette angle."""
    dims = (3, 2, 4, 2)
    lx, ly, lz, lt = dims
    rng = np.random.default_rng(3)
    theta = rng.uniform(-1, 1, size=(4, lt, lz, ly, lx))
    tdiag = np.array([1.0, -1.0, 0.0])
    u = np.zeros(sf.lattice_shape(dims) + (4, 3, 3), dtype=complex)
    for mu in range(4):
        u[..., mu, :, :] = np.exp(1j * theta[mu][..., None] * tdiag)[..., None] * np.eye(3)
    c = dirac.clover_field(u, 1.0)
    g, _ = cv.gammas()

    def th(mu, x, y, z, t):
        return theta[mu, t % lt, z % lz, y % ly, x % lx]

    def e(m):
        v = [0, 0, 0, 0]
        v[m] = 1
        return v

    for site in [(0, 0, 0, 0), (2, 1, 3, 1), (1, 0, 2, 1)]:
        want = np.zeros((4, 3, 4, 3), dtype=complex)
        for mu in range(4):
            for nu in range(mu + 1, 4):
                em, en = e(mu), e(nu)
                f = 0.0
                for cm, cn in [(0, 0), (-1, 0), (-1, -1), (0, -1)]:
                    m = [site[i] + cm * em[i] + cn * en[i] for i in range(4)]
                    mp = [m[i] + em[i] for i in range(4)]
                    mn = [m[i] + en[i] for i in range(4)]
                    phi = th(mu, *m) + th(nu, *mp) - th(mu, *mn) - th(nu, *m)
                    f += np.sin(phi) / 4.0
                sig = 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])
                want += -0.5 * np.einsum("st,ab->satb", sig, np.diag(f * tdiag))
        x, y, z, t = site
        np.testing.assert_allclose(c[t, z, y, x], want, atol=1e-14)


@pytest.mark.parametrize("kind,c_sw,anti", [("bri", 1.0, True), ("wil", 1.0, False), ("bri", 0.0, False)])
def test_per_site_oracle_matches_field_oracle(kind, c_sw, anti):
    """The per-site restatement used for sampled full-size checks agrees with the field oracle."""
    dims = (3, 4, 2, 3)
    u = sf.gauge_field(dims, 51)
    x = sf.gaussian_source(dims, 2, 52)
    op = dirac.DiracOperator(u, kind, m0=-0.8, c_sw=c_sw, antiperiodic_t=anti)
    full = op.apply(x)
    sites = [(0, 0, 0, 0), (2, 3, 1, 2), (1, 2, 0, 1), (2, 0, 1, 0)]
    got = dirac.apply_at_sites(u, kind, -0.8, c_sw, x, sites, antiperiodic_t=anti)
    for i, (sx, sy, sz, st) in enumerate(sites):
        np.testing.assert_allclose(got[:, i], full[:, st, sz, sy, sx], atol=1e-13)
