"""Seeded synthetic inputs: SU(3) gauge fields and Dirac sources.

Shared test/benchmark infrastructure.  Both the FP64 oracle checks and the CUDA
path read their inputs from here, so this module holds none of the overlap
method's arithmetic (no off-axis links, no Brillouin or Wilson stencil, no
Kenney-Laub rational, no solver).  It only manufactures inputs shaped like the
paper's workloads, which use thermalised quenched and N_f=2 ensembles (Sec. 6,
Sec. 8) that are not available here:

* links U_mu(n) = exp(i eps Q_mu(n)), Q = sum_a omega_a lambda_a / 2 with
  omega_a ~ N(0,1) drawn from numpy's PCG64 stream for ``seed``;
* optional isotropic stout smearing (Morningstar-Peardon), standing in for the
  paper's APE smearing of the kernel links;
* eps tuned by bisection so that the mean plaquette (1/3) Re tr P_{mu nu},
  measured after smearing, is 0.60 +- 0.005;
* complex Gaussian sources with Re, Im ~ N(0, 1/2) per component, or the 12
  spin-colour point sources at site 0.

Array conventions (a = 1):
  dims = (Lx, Ly, Lz, Lt); site index n = x + Lx*(y + Ly*(z + Lz*t));
  gauge field  U[t, z, y, x, mu, a, b]   complex128, mu = 0..3 <-> x, y, z, t;
  spinor field x[rhs, t, z, y, x, spin, colour] complex128.
"""
from __future__ import annotations

import functools

import numpy as np

__all__ = [
    "lattice_shape", "gauge_field", "tuned_eps", "plaquette", "stout_smear",
    "random_su3", "gaussian_source", "point_sources", "su3_exp_i",
]

TARGET_PLAQUETTE = 0.60


def lattice_shape(dims):
    """(Lt, Lz, Ly, Lx) array shape for dims = (Lx, Ly, Lz, Lt)."""
    lx, ly, lz, lt = (int(d) for d in dims)
    return (lt, lz, ly, lx)


def _gell_mann():
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


_LAMBDA = _gell_mann()


def su3_exp_i(h):
    """exp(i h) for a stack of Hermitian 3x3 matrices h (numpy or torch, via eigh)."""
    if _is_torch(h):
        return _expm_i_taylor(h)
    ev, vec = np.linalg.eigh(h)
    return np.einsum("...ab,...b,...cb->...ac", vec, np.exp(1j * ev), vec.conj())


def _expm_i_taylor(h, order=18):
    """exp(i h) by scaling and squaring with a truncated Taylor series
    (Moler & Van Loan): only batched matmuls, so it runs on any torch device.
    After scaling ||i h / 2^s||_F <= 1/2 the truncation error is below 1e-20."""
    import math

    import torch
    a = 1j * h
    nrm = float(torch.linalg.matrix_norm(a).max()) if a.numel() else 0.0
    sc = max(0, int(math.ceil(math.log2(max(nrm, 1e-300) / 0.5)))) if nrm > 0.5 else 0
    b = a / (2.0 ** sc)
    eye = torch.eye(3, dtype=h.dtype, device=h.device).expand_as(b)
    out = eye + b / order
    for k in range(order - 1, 0, -1):
        out = eye + (b @ out) / k
    for _ in range(sc):
        out = out @ out
    return out


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _shift(f, mu, s):
    """Field value at n + s*e_mu (periodic); f has leading axes (t, z, y, x)."""
    if _is_torch(f):
        import torch
        return torch.roll(f, -s, dims=3 - mu)
    return np.roll(f, -s, axis=3 - mu)


def _dag(m):
    if _is_torch(m):
        return m.transpose(-1, -2).conj()
    return np.swapaxes(m, -1, -2).conj()


def _trace(m):
    if _is_torch(m):
        return m.diagonal(dim1=-2, dim2=-1).sum(-1)
    return np.trace(m, axis1=-2, axis2=-1)


def plaquette(u):
    """Mean of (1/3) Re tr P_{mu nu}(n) over all sites and the 6 planes."""
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            um, un = u[..., mu, :, :], u[..., nu, :, :]
            p = um @ _shift(un, mu, 1) @ _dag(_shift(um, nu, 1)) @ _dag(un)
            tot += float(_trace(p).real.mean()) / 3.0
    return tot / 6.0


def stout_smear(u, rho, steps):
    """Isotropic stout smearing, ``steps`` sweeps with parameter ``rho``."""
    u = u.clone() if _is_torch(u) else u.copy()
    for _ in range(int(steps)):
        c = u * 0
        for mu in range(4):
            um = u[..., mu, :, :]
            for nu in range(4):
                if nu == mu:
                    continue
                un = u[..., nu, :, :]
                up = un @ _shift(um, nu, 1) @ _dag(_shift(un, mu, 1))
                un_m = _shift(un, nu, -1)
                dn = _dag(un_m) @ _shift(um, nu, -1) @ _shift(un_m, mu, 1)
                c[..., mu, :, :] += up + dn
        c = c * rho
        om = c @ _dag(u)
        a = _dag(om) - om
        tr = _trace(a)[..., None, None]
        if _is_torch(u):
            import torch
            eye = torch.eye(3, dtype=u.dtype, device=u.device)
        else:
            eye = np.eye(3)
        q = 0.5j * a - (1j / 6.0) * tr * eye
        q = 0.5 * (q + _dag(q))  # remove rounding-level anti-Hermitian part
        u = su3_exp_i(q) @ u
    return u


def _raw_field(shape, eps, rng, device=None):
    omega = rng.standard_normal(shape + (4, 8))
    if device is not None:
        import torch
        om = torch.from_numpy(omega).to(device)
        lam = torch.from_numpy(_LAMBDA).to(device)
        q = torch.einsum("...a,aij->...ij", om.to(torch.complex128), lam) * 0.5
        return su3_exp_i(eps * q)
    q = np.einsum("...a,aij->...ij", omega, _LAMBDA) * 0.5
    return su3_exp_i(eps * q)


@functools.lru_cache(maxsize=None)
def tuned_eps(smear_rho=0.0, smear_steps=0, target=TARGET_PLAQUETTE):
    """eps giving mean plaquette ``target`` (after smearing), tuned on 6^4.

    The plaquette of independent links is an intensive quantity, so the value
    tuned on a 6^4 lattice (fixed tuning seed) carries over to larger volumes.
    """
    shape = (6, 6, 6, 6)

    def plaq(eps):
        u = _raw_field(shape, eps, np.random.Generator(np.random.PCG64(987654321)))
        if smear_steps:
            u = stout_smear(u, smear_rho, smear_steps)
        return plaquette(u)

    lo, hi = 0.0, 4.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if plaq(mid) > target:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-4:
            break
    return 0.5 * (lo + hi)


def gauge_field(dims, seed, smear_rho=0.0, smear_steps=0, eps=None, device=None):
    """Seeded SU(3) field U[t,z,y,x,mu,3,3] (complex128 numpy), plaquette ~ 0.6.

    ``eps=0`` gives the free field U = 1.  ``device`` (e.g. "cuda") runs the
    matrix exponentials and smearing with torch on that device, for large
    volumes; the random numbers are the same numpy PCG64 stream either way,
    and the returned array is what both the oracle and the CUDA path consume.
    """
    shape = lattice_shape(dims)
    if eps is None:
        eps = tuned_eps(float(smear_rho), int(smear_steps))
    rng = np.random.Generator(np.random.PCG64(seed))
    u = _raw_field(shape, eps, rng, device)
    if smear_steps:
        u = stout_smear(u, smear_rho, smear_steps)
    if device is not None:
        u = u.cpu().numpy()
    return np.ascontiguousarray(u)


def random_su3(shape, seed):
    """Haar-ish random SU(3) matrices (QR of a complex Gaussian, det fixed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(tuple(shape) + (3, 3)) + 1j * rng.standard_normal(tuple(shape) + (3, 3))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    q = q / (det ** (1.0 / 3.0))[..., None, None]
    return q


def gaussian_source(dims, nrhs, seed, normalize=False):
    """Complex Gaussian spinors x[rhs,t,z,y,x,4,3], Re, Im ~ N(0, 1/2)."""
    shape = (int(nrhs),) + lattice_shape(dims) + (4, 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)
    if normalize:
        x /= np.sqrt((np.abs(x.reshape(nrhs, -1)) ** 2).sum(axis=1)).reshape((nrhs,) + (1,) * (x.ndim - 1))
    return x


def point_sources(dims, site=(0, 0, 0, 0)):
    """The 12 spin-colour point sources delta_{n,site} delta_{s,s0} delta_{c,c0}."""
    shape = (12,) + lattice_shape(dims) + (4, 3)
    x = np.zeros(shape, dtype=np.complex128)
    sx, sy, sz, st = site
    for s in range(4):
        for c in range(3):
            x[3 * s + c, st, sz, sy, sx, s, c] = 1.0
    return x
