"""Quality diagnostics (Sec. 5) and nested Kenney-Laub iterates (Sec. 4.1) on the
GPU through the C ABI, against the FP64 oracle:

* normality ||(D D^+ - D^+ D) eta|| and Ginsparg-Wilson defect
  ||(D g5 + g5 D - D g5 D / rho) eta|| of the massless overlap of order 1 (the
  f_11 operator of Sec. 5) and 4, Brillouin and Wilson kernels, c_SW = 1;
* the locality profile of D_ov eta for a single-site source (Sec. 5.3);
* the nested iterate D^(2) with orders (1, 1), which by g_3 o g_3 = g_9 = f_44
  equals the order-4 overlap, and (1, 2), equal to g_15 = f_77.
"""
import functools

import numpy as np
import pytest
import torch

import synthetic_fields as sf
from oracle import dirac, overlap
from oracle.dirac import gamma5
from paper_1701_00726_gb300 import Lattice

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


def _field():
    return sf.gauge_field(DIMS, 5, 0.1, 1)


@functools.lru_cache(maxsize=None)
def _oracle_defects(kind, n):
    u = _field()
    eta = sf.gaussian_source(DIMS, 2, 77, normalize=True)
    k = dirac.DiracOperator(u, kind, m0=-1.0, c_sw=1.0)

    def d(v):
        return overlap.overlap_apply(k, v, 1.0, n, 1e-13)[0]

    a0, a1 = d(eta), d(gamma5(eta))
    b0, b1 = d(gamma5(a0)), d(gamma5(a1))
    nm = [np.linalg.norm((b1 - gamma5(b0))[r]) for r in range(2)]
    gw = [np.linalg.norm((a1 + gamma5(a0) - b0)[r]) for r in range(2)]
    return nm, gw


@pytest.mark.parametrize("kind", ["bri", "wil"])
@pytest.mark.parametrize("n", [1, 4])
def test_normality_and_gw_defects_vs_oracle(kind, n):
    lat = Lattice(DIMS)
    lat.build_links(torch.from_numpy(_field()).cuda(), 1.0)
    lat.set_kernel(kind)
    eta = torch.from_numpy(sf.gaussian_source(DIMS, 2, 77, normalize=True)).cuda()
    nm, gw, st = lat.quality(eta, n, tol=1e-13)
    assert st["converged"]
    wnm, wgw = _oracle_defects(kind, n)
    for g, w in zip(nm + gw, wnm + wgw):
        assert abs(g - w) <= 1e-10 * max(1.0, w), (g, w)


def test_locality_profile_vs_oracle():
    dims = (6, 5, 4, 3)
    u = sf.gauge_field(dims, 6, 0.1, 3)
    src = 2 + dims[0] * (3 + dims[1] * (1 + dims[2] * 2))  # site (2, 3, 1, 2)
    rng = np.random.default_rng(5)
    eta = np.zeros((2,) + sf.lattice_shape(dims) + (4, 3), dtype=np.complex128)
    for r in range(2):
        v = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
        eta[r, 2, 1, 3, 2] = v / np.linalg.norm(v)
    nbins = 20
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    prof, counts, st = lat.locality(torch.from_numpy(eta).cuda(), src, 4, nbins, tol=1e-13)
    assert st["converged"]
    zeta, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), eta, 1.0, 4, 1e-13)
    want = np.zeros((2, nbins))
    wcnt = np.zeros(nbins, dtype=int)
    for t in range(dims[3]):
        for z in range(dims[2]):
            for y in range(dims[1]):
                for x in range(dims[0]):
                    r2 = 0
                    for c, s0, L in zip((x, y, z, t), (2, 3, 1, 2), dims):
                        d = abs(c - s0)
                        r2 += min(d, L - d) ** 2
                    if r2 < nbins:
                        wcnt[r2] += 1
                        want[:, r2] += np.linalg.norm(zeta[:, t, z, y, x].reshape(2, -1), axis=1)
    assert list(counts) == list(wcnt)
    assert np.abs(np.array(prof) - want).max() <= 1e-12 * np.abs(want).max()


@functools.lru_cache(maxsize=None)
def _oracle_overlap_ragged(n):
    dims = (6, 5, 4, 3)
    u = sf.gauge_field(dims, 7, 0.1, 3)
    x = sf.gaussian_source(dims, 1, 1017)
    want, _ = overlap.overlap_apply(dirac.DiracOperator(u, "bri", m0=-1.0, c_sw=1.0), x, 1.0, n, 1e-13)
    return want


@pytest.mark.parametrize("orders,equivalent", [((1, 1), 4), ((1, 2), 7)])
def test_nested_iterates(orders, equivalent):
    dims = (6, 5, 4, 3)
    u = sf.gauge_field(dims, 7, 0.1, 3)
    x = torch.from_numpy(sf.gaussian_source(dims, 1, 1017)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    y, st = lat.nested_apply(x, orders, tol=1e-13)
    assert st["converged"]
    y1, _ = lat.overlap_apply(x, equivalent, tol=1e-13)
    got = y.cpu().numpy()
    assert np.abs(got - y1.cpu().numpy()).max() <= 1e-10 * np.abs(got).max()
    want = _oracle_overlap_ragged(equivalent)
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
