"""ctypes binding of libtf.so: the C ABI declared in include/tf.h, same names.

This module only marshals arguments.  Every product runs in the library's CUDA
kernels; if the library is missing or cannot be loaded, ``lib()`` raises -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# TF_LIB_VARIANT=checked loads the bounds-checked debug build (libtf_checked.so);
# TF_LIB_PATH names any other build of the library (e.g. a tuning variant).
LIB_PATH = os.environ.get("TF_LIB_PATH") or os.path.join(
    HERE, "_build", "libtf_checked.so" if os.environ.get("TF_LIB_VARIANT") == "checked" else "libtf.so")

TF_OK, TF_EINVAL, TF_ENOMEM, TF_ECUDA, TF_EUNSUPPORTED, TF_ENOTCONV, TF_ETIMEOUT = range(7)
TF_F32, TF_F64 = 0, 1
STATUS_NAMES = {0: "TF_OK", 1: "TF_EINVAL", 2: "TF_ENOMEM", 3: "TF_ECUDA",
                4: "TF_EUNSUPPORTED", 5: "TF_ENOTCONV", 6: "TF_ETIMEOUT"}


class tf_grid(ctypes.Structure):
    _fields_ = [("sx", ctypes.c_int), ("sy", ctypes.c_int), ("nz", ctypes.c_int),
                ("pxl", ctypes.c_int), ("pxr", ctypes.c_int), ("pyl", ctypes.c_int),
                ("pyr", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("z_edges", ctypes.POINTER(ctypes.c_double)), ("station_z", ctypes.c_double)]


class tf_irls_params(ctypes.Structure):
    _fields_ = [("t", ctypes.c_int), ("tp", ctypes.c_int), ("beta", ctypes.c_double),
                ("lam", ctypes.c_double), ("eps2", ctypes.c_double), ("lower", ctypes.c_double),
                ("upper", ctypes.c_double), ("kmax", ctypes.c_int), ("chi2_stop", ctypes.c_int),
                ("reorth", ctypes.c_int), ("alphas", ctypes.POINTER(ctypes.c_double))]


class tf_irls_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("chi2", ctypes.POINTER(ctypes.c_double)),
                ("seconds", ctypes.POINTER(ctypes.c_double))]


class tf_batch_opts(ctypes.Structure):
    _fields_ = [("rows_tile", ctypes.c_int), ("cols_tile", ctypes.c_int), ("claim", ctypes.c_int),
                ("wait_ms", ctypes.c_double), ("gate", ctypes.c_void_p),
                ("use_graph", ctypes.c_int)]


class TFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

vp = ctypes.c_void_p
i64 = ctypes.c_int64
c_int = ctypes.c_int
P = ctypes.POINTER

SIGNATURES = {
    "tf_create_gravity": [P(tf_grid), c_int, vp, P(vp)],
    "tf_create_magnetic": [P(tf_grid), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           c_int, vp, P(vp)],
    "tf_destroy": [vp],
    "tf_dims": [vp, P(i64), P(i64)],
    "tf_fft_dims": [vp, P(c_int), P(c_int)],
    "tf_matvec": [vp, vp, vp, vp, vp, vp],
    "tf_rmatvec": [vp, vp, vp, vp, vp, vp],
    "tf_matmat": [vp, i64, vp, i64, vp, i64, vp, vp, vp],
    "tf_rmatmat": [vp, i64, vp, i64, vp, i64, vp, vp, vp],
    "tf_get_spectra": [vp, vp, i64, vp],
    "tf_products_host": [vp, i64, vp, i64, vp, i64, i64, vp, i64, vp, i64, vp, vp, c_int, vp],
    "tf_set_tuning": [vp, c_int, c_int, i64],
    "tf_get_tuning": [vp, P(c_int), P(c_int), P(i64)],
    "tf_profile_enable": [vp, c_int],
    "tf_profile_read": [vp, P(ctypes.c_double), P(i64), P(i64)],
    "tf_matvec_noalloc": [vp, vp, vp, vp, vp, vp],
    "tf_set_engine": [vp, c_int],
    "tf_get_engine": [vp, P(c_int), P(c_int), P(c_int)],
    "tf_debug_oob": [P(c_int), P(c_int), P(i64), P(i64)],
    "tf_peak_probe": [c_int, P(ctypes.c_double), vp],
    "tf_rows_dot": [c_int, vp, i64, i64, i64, vp, vp, vp],
    "tf_rows_axpy": [c_int, vp, i64, i64, i64, vp, vp, vp],
    "tf_gkb": [vp, P(tf_irls_params), vp, vp, vp, P(tf_irls_report), vp],
    "tf_rsvd": [vp, P(tf_irls_params), vp, vp, vp, vp, P(tf_irls_report), vp],
    "tf_tridiag_eig_first": [c_int, vp, vp, vp],
    "tf_batch_create": [P(vp), c_int, c_int, P(vp)],
    "tf_batch_destroy": [vp],
    "tf_batch_products": [vp, i64, P(vp), P(vp), P(vp), P(vp), c_int, vp],
    "tf_damped_bidiag_solve": [c_int, vp, vp, ctypes.c_double, ctypes.c_double, vp],
    "tf_batch_persistent": [vp, i64, P(vp), P(vp), P(vp), P(vp), P(tf_batch_opts), vp],
    "tf_set_radices": [vp, c_int, P(c_int), c_int],
    "tf_get_radices": [vp, c_int, P(c_int), P(c_int)],
}


def lib():
    """Load libtf.so (built in-tree by ``paper_2004_13904_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2004_13904_gb300.build` (no CPU fallback exists)")
    L = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = c_int
    L.tf_last_error.argtypes = []
    L.tf_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


def check(status: int) -> None:
    if status != TF_OK:
        raise TFError(status, lib().tf_last_error().decode(errors="replace"))


def make_grid(g):
    """tf_grid from any object with sx, sy, nz, pxl, pxr, pyl, pyr, dx, dy, z_edges,
    station_z attributes; returns (struct, keepalive array)."""
    z = (ctypes.c_double * (g.nz + 1))(*[float(v) for v in g.z_edges])
    s = tf_grid(int(g.sx), int(g.sy), int(g.nz), int(g.pxl), int(g.pxr), int(g.pyl),
                int(g.pyr), float(g.dx), float(g.dy), ctypes.cast(z, P(ctypes.c_double)),
                float(g.station_z))
    return s, z
