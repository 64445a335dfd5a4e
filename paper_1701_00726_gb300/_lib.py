"""ctypes binding of libbri.so: argument marshalling only.

Every function here forwards to the C ABI declared in include/bri.h with the
same name; all arithmetic runs in the library's CUDA kernels.  Tensors are
passed as raw device pointers (``tensor.data_ptr()``); the binding checks
dtype, device, contiguity and size so that a wrong tensor fails in Python
instead of reaching the kernels.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbri.so")

BRI_OK = 0
BRI_NOT_CONVERGED = 1
PREC_F64 = 0
PREC_F32 = 1
PREC_F32_BF16 = 2
PREC_DW = 3  # bri_apply only: complex128 in/out, double-word FP32 arithmetic
ANTIPERIODIC_T = 1
KERNEL_BRILLOUIN = 0
KERNEL_WILSON = 1
KL_DIAGONAL = 0
KL_UPPER = 1
MAX_SHIFTS = 32


class BriStats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("matvecs", ctypes.c_int),
        ("matvecs_f64", ctypes.c_int),
        ("refinements", ctypes.c_int),
        ("n_shifts", ctypes.c_int),
        ("max_true_residual", ctypes.c_double),
        ("shift_residual", ctypes.c_double * MAX_SHIFTS),
        ("want_true_residual", ctypes.c_int),
        ("maxiter", ctypes.c_int),
        ("seconds", ctypes.c_double),
        ("phase_seconds", ctypes.c_double * 4),
    ]

    def as_dict(self):
        return {
            "iterations": self.iterations, "matvecs": self.matvecs, "matvecs_f64": self.matvecs_f64,
            "refinements": self.refinements, "n_shifts": self.n_shifts,
            "max_true_residual": self.max_true_residual,
            "shift_residual": list(self.shift_residual)[: self.n_shifts], "seconds": self.seconds,
            "phase_seconds": list(self.phase_seconds),
        }


class BriError(RuntimeError):
    pass


_lib = None

_SIGS = {
    "bri_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  ctypes.c_void_p]),
    "bri_destroy": (None, [ctypes.c_void_p]),
    "bri_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bri_set_kernel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bri_build_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    "bri_get_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "bri_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_int]),
    "wils_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_int]),
    "kl_coeffs": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "sign_apply_multishift": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, ctypes.POINTER(BriStats)]),
    "overlap_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(BriStats)]),
    "overlap_apply_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.POINTER(BriStats)]),
    "overlap_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(BriStats)]),
    "overlap_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(BriStats)]),
    "sign_apply_multishift_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_double, ctypes.POINTER(BriStats)]),
    "bri_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bri_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "overlap_quality": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(BriStats)]),
    "overlap_locality": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(BriStats)]),
    "overlap_nested_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                                            ctypes.c_double, ctypes.POINTER(BriStats)]),
    "bri_dispersion": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "bri_fma_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "bri_kernel_launches": (ctypes.c_longlong, []),
    "bri_device_allocations": (ctypes.c_longlong, []),
    "bri_last_error": (ctypes.c_char_p, []),
}

EXPORTED = tuple(_SIGS)


def load(path=LIB_PATH):
    """Load libbri.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise BriError(f"{path} not found: build the CUDA library first (python -c 'import __graft_entry__ as g; "
                       "g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(rc, what):
    if rc < 0:
        raise BriError(f"{what} failed ({rc}): {load().bri_last_error().decode()}")
    return rc


def dispersion(momenta, masses, kernel=KERNEL_BRILLOUIN, overlap=False, rho=1.0, stream=0):
    """Free-field energies aE for spatial momenta [(p1, p2, p3), ...] and masses am (Sec. 2, App. A)."""
    lib = load()
    n = len(masses)
    if n == 0 or len(momenta) != n:
        raise BriError("dispersion: need one mass per momentum")
    p = (ctypes.c_double * (3 * n))(*[float(c) for q in momenta for c in q])
    m = (ctypes.c_double * n)(*[float(v) for v in masses])
    e = (ctypes.c_double * n)()
    check(lib.bri_dispersion(int(kernel), int(bool(overlap)), float(rho), n, p, m, e, ctypes.c_void_p(stream)),
          "bri_dispersion")
    return list(e)


def fma_probe(kind, stream=0):
    """(TFLOP/s, ms) of the FMA-throughput probe: kind 0 FP64, 1 FP32, 2 paired FP32."""
    lib = load()
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    check(lib.bri_fma_probe(int(kind), ctypes.c_void_p(stream), ctypes.byref(tf), ctypes.byref(ms)), "bri_fma_probe")
    return tf.value, ms.value


def kl_coeffs(n, kind=KL_DIAGONAL, scale=1.0):
    lib = load()
    c0 = ctypes.c_double()
    w = (ctypes.c_double * n)()
    s = (ctypes.c_double * n)()
    check(lib.kl_coeffs(n, kind, scale, ctypes.byref(c0), w, s), "kl_coeffs")
    return c0.value, list(w), list(s)
