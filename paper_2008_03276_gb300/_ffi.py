"""ctypes view of the C ABI in ``include/ehl.h`` (argument marshalling only).

The shared library is loaded from ``_lib/libehl_gb300.so`` next to this file.
There is no fallback: if the library is missing or cannot be loaded, every
entry point raises.
"""
import ctypes
import os

from . import build as _build

class EhlParams(ctypes.Structure):
    """Mirror of ``ehl_params`` in include/ehl.h (same field order and types)."""

    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("xa", ctypes.c_double), ("xb", ctypes.c_double), ("ya", ctypes.c_double), ("yb", ctypes.c_double),
                ("M", ctypes.c_double), ("L", ctypes.c_double), ("alpha", ctypes.c_double),
                ("p0", ctypes.c_double), ("z", ctypes.c_double),
                ("compressible", ctypes.c_int), ("elastic", ctypes.c_int), ("limiter", ctypes.c_int),
                ("halfband", ctypes.c_int), ("switch_eps_h", ctypes.c_double), ("dist_weight", ctypes.c_double),
                ("c_h0", ctypes.c_double), ("omega", ctypes.c_double), ("method", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("krylov_dim", ctypes.c_int),
                ("h_init", ctypes.c_double), ("levels", ctypes.c_int), ("coarse_min_nodes", ctypes.c_int),
                ("coarse_tol", ctypes.c_double), ("precond_blocks", ctypes.c_int),
                ("precision", ctypes.c_int), ("graph", ctypes.c_int), ("kappa", ctypes.c_double),
                ("splitting", ctypes.c_int), ("deform", ctypes.c_int), ("autotune", ctypes.c_int), ("yline", ctypes.c_int)]


class EhlCdParams(ctypes.Structure):
    """Mirror of ``ehl_cd_params`` in include/ehl.h."""

    _fields_ = [("n", ctypes.c_int), ("lo", ctypes.c_double), ("hi", ctypes.c_double), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("eps", ctypes.c_double), ("kappa", ctypes.c_double),
                ("splitting", ctypes.c_int), ("order", ctypes.c_int), ("omega", ctypes.c_double)]


EHL_OK, EHL_EINVAL, EHL_ENOMEM, EHL_ECUDA, EHL_ENOCONV, EHL_ENONFINITE, EHL_ESINGULAR, EHL_ETIMEOUT = range(8)

# every symbol the header declares; the CPU tests check the library exports them
SYMBOLS = {
    "ehl_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "ehl_version": (ctypes.c_int, []),
    "ehl_kernel_launches": (ctypes.c_ulonglong, []),
    "ehl_paqif_workspace_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "ehl_paqif_solve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ehl_paqif_workspace_size_partitioned": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                            ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "ehl_paqif_partitions": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_int)]),
    "ehl_paqif_solve_partitioned": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                   ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "ehl_params_default": (None, [ctypes.POINTER(EhlParams), ctypes.c_int]),
    "ehl_create": (ctypes.c_int, [ctypes.POINTER(EhlParams), ctypes.c_int, ctypes.POINTER(EhlParams),
                                  ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "ehl_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "ehl_adjoint": (ctypes.c_int, [ctypes.c_void_p] * 10 + [ctypes.c_double, ctypes.c_int]),
    "ehl_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ehl_jacobian_band": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "ehl_jacobian_apply": (ctypes.c_int, [ctypes.c_void_p] * 7),
    "ehl_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p]),
    "ehl_cd_residual": (ctypes.c_int, [ctypes.POINTER(EhlCdParams), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ehl_cd_workspace_size": (ctypes.c_int, [ctypes.POINTER(EhlCdParams), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "ehl_cd_relax": (ctypes.c_int, [ctypes.POINTER(EhlCdParams), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p]),
    "ehl_paqif_autotune": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "ehl_paqif_factor_size": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "ehl_paqif_factor": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_size_t, ctypes.c_void_p]),
    "ehl_paqif_resolve": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "ehl_paqif_solve_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}

_lib = None


class EhlError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {status_string(code)}")


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) and return the ctypes library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"EHL CUDA library not found at {path}; run paper_2008_03276_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(code):
    return load().ehl_status_string(int(code)).decode()


def check(code, where):
    if code != EHL_OK:
        raise EhlError(code, where)
