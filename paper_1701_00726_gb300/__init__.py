"""GB300-native Brillouin-kernel overlap operator (arXiv:1701.00726).

The compute path is the CUDA library ``libbri.so`` behind the C ABI of
``include/bri.h``; this package only marshals PyTorch tensors (device memory
and streams) into it.  There is no CPU fallback: importing works without a
GPU, but every operator call needs the built library and a CUDA device.

Spinors are complex tensors of shape ``[nrhs, Lt, Lz, Ly, Lx, 4, 3]`` (or any
shape with ``nrhs * V * 12`` elements, C-contiguous), complex128 for the FP64
path and complex64 for the FP32 / BF16-link paths; gauge fields are complex128
``[Lt, Lz, Ly, Lx, 4, 3, 3]``.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (ANTIPERIODIC_T, BRI_NOT_CONVERGED, KERNEL_BRILLOUIN, KERNEL_WILSON, KL_DIAGONAL, KL_UPPER,
                   PREC_DW, PREC_F32, PREC_F32_BF16, PREC_F64, BriError, BriStats, dispersion, kl_coeffs)

__all__ = ["Lattice", "overlap", "OverlapFunction", "overlap_apply_batch", "kl_coeffs", "dispersion", "BriError",
           "BriStats",
           "PREC_F64", "PREC_F32", "PREC_F32_BF16", "PREC_DW", "KL_DIAGONAL", "KL_UPPER", "ANTIPERIODIC_T", "KERNEL_BRILLOUIN",
           "KERNEL_WILSON"]


def _torch():
    import torch
    return torch


class Lattice:
    """One lattice (dims = (Lx, Ly, Lz, Lt)) with its links, on the current CUDA device."""

    def __init__(self, dims, antiperiodic_t=False, stream=None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise BriError("a CUDA device is required (libbri has no CPU path)")
        self.lib = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.volume = self.dims[0] * self.dims[1] * self.dims[2] * self.dims[3]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        handle = ctypes.c_void_p()
        arr = (ctypes.c_int * 4)(*self.dims)
        flags = ANTIPERIODIC_T if antiperiodic_t else 0
        _lib.check(self.lib.bri_create(ctypes.byref(handle), arr, flags, ctypes.c_void_p(self.stream.cuda_stream)),
                   "bri_create")
        self._h = handle

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.bri_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ marshalling helpers
    def _spinor(self, x, dtypes):
        torch = _torch()
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise BriError("spinor must be a CUDA tensor")
        if x.dtype not in dtypes:
            raise BriError(f"spinor dtype {x.dtype} not in {dtypes}")
        if not x.is_contiguous():
            raise BriError("spinor must be contiguous")
        per = self.volume * 12
        if x.numel() == 0 or x.numel() % per:
            raise BriError(f"spinor has {x.numel()} elements, not a multiple of V*12 = {per}")
        return x.numel() // per

    def build_links(self, u, c_sw=0.0):
        torch = _torch()
        if u.dtype != torch.complex128 or not u.is_cuda or not u.is_contiguous():
            raise BriError("gauge field must be a contiguous complex128 CUDA tensor")
        if u.numel() != self.volume * 36:
            raise BriError("gauge field must have V*4*3*3 elements")
        _lib.check(self.lib.bri_build_links(self._h, ctypes.c_void_p(u.data_ptr()), float(c_sw)), "bri_build_links")

    def set_kernel(self, kernel):
        """Kernel operator of the overlap solvers: KERNEL_BRILLOUIN ("bri") or KERNEL_WILSON ("wil")."""
        k = {"bri": KERNEL_BRILLOUIN, "wil": KERNEL_WILSON}.get(kernel, kernel)
        _lib.check(self.lib.bri_set_kernel(self._h, int(k)), "bri_set_kernel")

    def links(self):
        """Stored off-axis links, complex128 [V, 40, 3, 3] (App. C layout)."""
        torch = _torch()
        w = torch.empty((self.volume, 40, 3, 3), dtype=torch.complex128, device="cuda")
        _lib.check(self.lib.bri_get_links(self._h, ctypes.c_void_p(w.data_ptr())), "bri_get_links")
        return w

    def profile(self, enable=True):
        _lib.check(self.lib.bri_profile_enable(self._h, int(bool(enable))), "bri_profile_enable")

    def profile_read(self, op=0, prec=PREC_F32):
        """(launches, kernel ms, site*rhs units) of one stencil since the last read."""
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        units = ctypes.c_double()
        _lib.check(self.lib.bri_profile_read(self._h, int(op), int(prec), ctypes.byref(n), ctypes.byref(ms),
                                             ctypes.byref(units)), "bri_profile_read")
        return n.value, ms.value, units.value

    @staticmethod
    def kernel_launches():
        return int(_lib.load().bri_kernel_launches())

    @staticmethod
    def device_allocations():
        return int(_lib.load().bri_device_allocations())

    @staticmethod
    def _prec_for(x, bf16_links):
        torch = _torch()
        if x.dtype == torch.complex128:
            return PREC_F64
        return PREC_F32_BF16 if bf16_links else PREC_F32

    def bri_apply(self, x, m0, dagger=False, bf16_links=False, out=None, double_word=False):
        """y = D_bri x (or D^dagger x).  complex128 x: FP64, or with double_word=True the double-word
        FP32 operator (FP64-class accuracy on the FP32 pipe); complex64 x: FP32 (or BF16-stored) links."""
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128, torch.complex64))
        if double_word and x.dtype != torch.complex128:
            raise BriError("bri_apply: the double-word operator takes complex128 spinors")
        y = torch.empty_like(x) if out is None else out
        prec = PREC_DW if double_word else self._prec_for(x, bf16_links)
        _lib.check(self.lib.bri_apply(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs,
                                      float(m0), int(bool(dagger)), prec), "bri_apply")
        return y

    def wils_apply(self, x, m0, dagger=False, out=None):
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128, torch.complex64))
        y = torch.empty_like(x) if out is None else out
        _lib.check(self.lib.wils_apply(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs,
                                       float(m0), int(bool(dagger)), self._prec_for(x, False)), "wils_apply")
        return y

    def _solver_stats(self, want_true_residual, maxiter):
        st = BriStats()
        st.want_true_residual = int(bool(want_true_residual))
        st.maxiter = int(maxiter)
        return st

    def sign_apply(self, x, n, rho=1.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL, scale=1.0,
                   want_true_residual=False, maxiter=0, out=None):
        """gamma5 f_nn(H) x, H = gamma5 D_bri(-rho); x complex128.  Returns (y, stats)."""
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128,))
        y = torch.empty_like(x) if out is None else out
        st = self._solver_stats(want_true_residual, maxiter)
        rc = self.lib.sign_apply_multishift(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                            nrhs, int(n), int(kind), float(rho), float(scale), float(tol), int(prec),
                                            ctypes.byref(st))
        _lib.check(rc, "sign_apply_multishift")
        d = st.as_dict()
        d["converged"] = rc == 0
        return y, d

    def overlap_solve(self, b, n_outer, n_inner=0, rho=1.0, am=0.0, complete=True, tol=1e-12, prec=PREC_F64,
                      kind=KL_DIAGONAL, maxiter=0, out=None):
        """Solve D_m x = b (traditional or complete massive overlap) by BiCGstab with the
        cascaded preconditioner of order n_inner (0: none).  Returns (x, stats)."""
        torch = _torch()
        nrhs = self._spinor(b, (torch.complex128,))
        x = torch.empty_like(b) if out is None else out
        st = self._solver_stats(False, maxiter)
        rc = self.lib.overlap_solve(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(b.data_ptr()), nrhs,
                                    int(n_outer), int(n_inner), int(kind), float(rho), float(am), int(bool(complete)),
                                    float(tol), int(prec), ctypes.byref(st))
        _lib.check(rc, "overlap_solve")
        d = st.as_dict()
        d["converged"] = rc == 0
        return x, d

    def overlap_grad(self, eta, psi, n, rho=1.0, am=0.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL, scale=1.0,
                     maxiter=0):
        """Adjoint of overlap_apply for L = sum_r Re<eta_r, D_m psi_r>: returns (g_psi, g_U, stats),
        g_U with the shape [Lt, Lz, Ly, Lx, 4, 3, 3] of the gauge field (through the off-axis links
        or, for the Wilson kernel, the thin links, and the clover term when c_sw != 0)."""
        torch = _torch()
        nrhs = self._spinor(psi, (torch.complex128,))
        if self._spinor(eta, (torch.complex128,)) != nrhs:
            raise BriError("eta and psi must hold the same number of right-hand sides")
        g_psi = torch.empty_like(psi)
        lt, lz, ly, lx = self.dims[3], self.dims[2], self.dims[1], self.dims[0]
        g_u = torch.empty((lt, lz, ly, lx, 4, 3, 3), dtype=torch.complex128, device=psi.device)
        st = self._solver_stats(False, maxiter)
        rc = self.lib.overlap_grad(self._h, ctypes.c_void_p(g_psi.data_ptr()), ctypes.c_void_p(g_u.data_ptr()),
                                   ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(psi.data_ptr()), nrhs, int(n),
                                   int(kind), float(rho), float(am), float(scale), float(tol), int(prec),
                                   ctypes.byref(st))
        _lib.check(rc, "overlap_grad")
        d = st.as_dict()
        d["converged"] = rc == 0
        return g_psi, g_u, d

    def sign_apply_noalloc(self, x, n, rho=1.0, tol=1e-12, kind=KL_DIAGONAL, scale=1.0, out=None):
        """FP64 gamma5 f_nn(H) x through the entry point that allocates no device memory
        (its workspace is a fixed 32 MiB device array).  ``out`` lets the caller keep
        allocation out of this call too.  Returns (y, stats)."""
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128,))
        y = torch.empty_like(x) if out is None else out
        st = self._solver_stats(False, 0)
        rc = self.lib.sign_apply_multishift_noalloc(self._h, ctypes.c_void_p(y.data_ptr()),
                                                    ctypes.c_void_p(x.data_ptr()), nrhs, int(n), int(kind),
                                                    float(rho), float(scale), float(tol), ctypes.byref(st))
        _lib.check(rc, "sign_apply_multishift_noalloc")
        d = st.as_dict()
        d["converged"] = rc == 0
        return y, d

    def quality(self, eta, n, rho=1.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL):
        """Normality and Ginsparg-Wilson defects ||(D D^+ - D^+ D) eta||, ||(D g5 + g5 D - D g5 D / rho) eta||
        of the massless overlap of order n, per source (Sec. 5).  Returns (normality, gw, stats)."""
        torch = _torch()
        nrhs = self._spinor(eta, (torch.complex128,))
        nm = (ctypes.c_double * nrhs)()
        gw = (ctypes.c_double * nrhs)()
        st = self._solver_stats(False, 0)
        rc = self.lib.overlap_quality(self._h, ctypes.c_void_p(eta.data_ptr()), nrhs, int(n), int(kind), float(rho),
                                      float(tol), int(prec), nm, gw, ctypes.byref(st))
        _lib.check(rc, "overlap_quality")
        d = st.as_dict()
        d["converged"] = rc == 0
        return list(nm), list(gw), d

    def locality(self, eta, src, n, nbins, rho=1.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL):
        """Sec. 5.3: per source, the sum of |D_ov eta (x)| over sites with |x - src|^2 = b, b < nbins,
        and the number of such sites.  ``src`` is a site index.  Returns (profile[nrhs][nbins], counts, stats)."""
        torch = _torch()
        nrhs = self._spinor(eta, (torch.complex128,))
        prof = (ctypes.c_double * (nrhs * nbins))()
        cnt = (ctypes.c_int * nbins)()
        st = self._solver_stats(False, 0)
        rc = self.lib.overlap_locality(self._h, ctypes.c_void_p(eta.data_ptr()), nrhs, int(src), int(n), int(kind),
                                       float(rho), float(tol), int(prec), int(nbins), prof, cnt, ctypes.byref(st))
        _lib.check(rc, "overlap_locality")
        d = st.as_dict()
        d["converged"] = rc == 0
        p = [list(prof[r * nbins:(r + 1) * nbins]) for r in range(nrhs)]
        return p, list(cnt), d

    def nested_apply(self, x, orders, rho=1.0, tol=1e-12, out=None):
        """D^(k) x = rho (x + Y_k x) with the nested Kenney-Laub iterates of the given orders (Sec. 4.1)."""
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128,))
        y = torch.empty_like(x) if out is None else out
        orders = [int(v) for v in orders]
        arr = (ctypes.c_int * len(orders))(*orders)
        st = self._solver_stats(False, 0)
        rc = self.lib.overlap_nested_apply(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                           nrhs, len(orders), arr, float(rho), float(tol), ctypes.byref(st))
        _lib.check(rc, "overlap_nested_apply")
        d = st.as_dict()
        d["converged"] = rc == 0
        return y, d

    def overlap_apply(self, x, n, rho=1.0, am=0.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL, scale=1.0,
                      want_true_residual=False, maxiter=0, out=None):
        """(1 - am/(2 rho)) D_ov x + am x with D_ov = rho (1 + gamma5 f_nn(H)).  Returns (y, stats)."""
        torch = _torch()
        nrhs = self._spinor(x, (torch.complex128,))
        y = torch.empty_like(x) if out is None else out
        st = self._solver_stats(want_true_residual, maxiter)
        rc = self.lib.overlap_apply(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), nrhs,
                                    int(n), int(kind), float(rho), float(am), float(scale), float(tol), int(prec),
                                    ctypes.byref(st))
        _lib.check(rc, "overlap_apply")
        d = st.as_dict()
        d["converged"] = rc == 0
        return y, d


def overlap_apply_batch(lattices, xs, n, rho=1.0, am=0.0, tol=1e-12, prec=PREC_F64, kind=KL_DIAGONAL, scale=1.0):
    """overlap_apply on several independent lattices at once (concurrently on the GPU).
    Returns (list of y, list of stats)."""
    torch = _torch()
    k = len(lattices)
    if k != len(xs) or k == 0:
        raise BriError("need one source tensor per lattice")
    lib = _lib.load()
    nrhs = [lat._spinor(x, (torch.complex128,)) for lat, x in zip(lattices, xs)]
    ys = [torch.empty_like(x) for x in xs]
    for lat in lattices:  # the batch runs after everything already queued on the callers' streams
        lat.stream.synchronize()
    ctxs = (ctypes.c_void_p * k)(*[lat._h.value for lat in lattices])
    yp = (ctypes.c_void_p * k)(*[y.data_ptr() for y in ys])
    xp = (ctypes.c_void_p * k)(*[x.data_ptr() for x in xs])
    nr = (ctypes.c_int * k)(*nrhs)
    sts = (BriStats * k)()
    rc = lib.overlap_apply_batch(ctxs, k, yp, xp, nr, int(n), int(kind), float(rho), float(am), float(scale),
                                 float(tol), int(prec), sts)
    _lib.check(rc, "overlap_apply_batch")
    out = []
    for i in range(k):
        d = sts[i].as_dict()
        out.append(d)
    return ys, out


class OverlapFunction:
    """torch.autograd.Function for y = D_m psi with gradients for psi and the gauge field.

    Built lazily so that importing the package does not import torch.
    """

    _fn = None

    @classmethod
    def get(cls):
        if cls._fn is None:
            torch = _torch()

            class _Overlap(torch.autograd.Function):
                @staticmethod
                def forward(ctx, psi, u, lattice, n, rho, am, tol, prec, c_sw):
                    lattice.build_links(u.detach().contiguous(), c_sw)
                    y, _ = lattice.overlap_apply(psi.detach().contiguous(), n, rho=rho, am=am, tol=tol, prec=prec)
                    ctx.save_for_backward(psi.detach())
                    ctx.cfg = (lattice, n, rho, am, tol, prec)
                    return y

                @staticmethod
                def backward(ctx, grad_y):
                    (psi,) = ctx.saved_tensors
                    lattice, n, rho, am, tol, prec = ctx.cfg
                    g_psi, g_u, _ = lattice.overlap_grad(grad_y.contiguous(), psi, n, rho=rho, am=am, tol=tol,
                                                         prec=prec)
                    return g_psi, g_u, None, None, None, None, None, None, None

            cls._fn = _Overlap
        return cls._fn


def overlap(psi, u, lattice, n, rho=1.0, am=0.0, tol=1e-12, prec=PREC_F64, c_sw=0.0):
    """Differentiable D_m psi = (1 - am/(2 rho)) D_ov psi + am psi, with the lattice's kernel
    (links and clover term rebuilt from ``u`` with coefficient ``c_sw``)."""
    return OverlapFunction.get().apply(psi, u, lattice, n, rho, am, tol, prec, c_sw)
