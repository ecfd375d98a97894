"""GB300-native BTTB/BCCB sensitivity products for fast focusing inversion.

``Operator`` wraps one tf_op of libtf.so (include/tf.h): the layer spectra of a gravity
or magnetic sensitivity matrix G, and the products G X, G^T Y on CUDA tensors.  PyTorch
provides device memory and streams only; every step of a product runs in the
library's kernels.
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import TFError, TF_F32, TF_F64  # noqa: F401

__all__ = ["Operator", "TFError", "STAGES", "peak_tflops"]

STAGES = ("rows_r2c_model", "cols_fwd", "rows_c2r_data",
          "rows_r2c_data", "cols_adj", "rows_c2r_model")


def _torch():
    import torch
    return torch


def peak_tflops(dtype) -> float:
    """Measured FMA throughput (TFLOP/s) of the current GPU for torch.float32/float64."""
    torch = _torch()
    v = ctypes.c_double()
    dt = TF_F32 if dtype == torch.float32 else TF_F64
    _lib.check(_lib.lib().tf_peak_probe(dt, ctypes.byref(v),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return v.value


class Operator:
    """G for one station/volume geometry (Sec. 2.1), applied by 2-D FFTs (App. A).

    grid: object with sx, sy, nz, pxl, pxr, pyl, pyr, dx, dy, z_edges, station_z.
    kind: "gravity" (mGal per g/cc) or "magnetic" (nT per SI, needs inc/dec in degrees).
    dtype: torch.float32 (FP32 spectra and FFTs) or torch.float64 (plain FP64 path).
    """

    def __init__(self, grid, kind: str = "gravity", inc: float = 90.0, dec: float = 0.0,
                 field_nt: float = 50000.0, dtype=None, device=None):
        torch = _torch()
        self.dtype = torch.float32 if dtype is None else dtype
        if self.dtype not in (torch.float32, torch.float64):
            raise ValueError("dtype must be torch.float32 or torch.float64")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        L = _lib.lib()
        gs, self._z = _lib.make_grid(grid)
        dt = TF_F32 if self.dtype == torch.float32 else TF_F64
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
            if kind == "gravity":
                _lib.check(L.tf_create_gravity(ctypes.byref(gs), dt, stream, ctypes.byref(h)))
            elif kind == "magnetic":
                _lib.check(L.tf_create_magnetic(ctypes.byref(gs), float(inc), float(dec),
                                                float(field_nt), dt, stream, ctypes.byref(h)))
            else:
                raise ValueError(f"unknown kind {kind!r}")
        self._h = h
        self.kind = kind
        m = ctypes.c_int64()
        n = ctypes.c_int64()
        _lib.check(L.tf_dims(h, ctypes.byref(m), ctypes.byref(n)))
        self.m, self.n = m.value, n.value
        n1 = ctypes.c_int()
        n2 = ctypes.c_int()
        _lib.check(L.tf_fft_dims(h, ctypes.byref(n1), ctypes.byref(n2)))
        self.n1, self.n2 = n1.value, n2.value
        self.nz = int(grid.nz)

    # -- plumbing -----------------------------------------------------------------------
    def close(self):
        """Frees the operator; raises TFError when tf_destroy reports a fault of pending work
        or a device-side wait that ran out (TF_ETIMEOUT)."""
        if getattr(self, "_h", None):
            h, self._h = self._h, None
            _lib.check(_lib.lib().tf_destroy(h))

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    def _vec(self, t, length, name):
        torch = _torch()
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype:
            raise TypeError(f"{name} must be a {self.dtype} tensor on {self.device}")
        if t.numel() != length or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with {length} elements")
        return t

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)

    def _block(self, t, rows, name):
        """(B, rows) tensor whose row b is column b of a column-major block."""
        torch = _torch()
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != self.dtype:
            raise TypeError(f"{name} must be a {self.dtype} tensor on {self.device}")
        if t.dim() == 1:
            t = t.view(1, -1)
        if t.dim() != 2 or t.shape[1] != rows or t.stride(1) != 1 or (
                t.shape[0] > 1 and t.stride(0) < rows):
            raise ValueError(f"{name} must have shape (B, {rows}) with unit inner stride")
        return t, (t.stride(0) if t.shape[0] > 1 else rows)

    # -- products -----------------------------------------------------------------------
    def matmat(self, X, colscale=None, rowscale=None, out=None):
        """D = diag(rowscale) G diag(colscale) X; X is (B, n), result (B, m)."""
        torch = _torch()
        X, ldx = self._block(X, self.n, "X")
        B = X.shape[0]
        if out is None:
            out = torch.empty((B, self.m), device=self.device, dtype=self.dtype)
        D, ldd = self._block(out, self.m, "out")
        cs = self._vec(colscale, self.n, "colscale")
        rs = self._vec(rowscale, self.m, "rowscale")
        _lib.check(_lib.lib().tf_matmat(self._h, B, self._ptr(X), ldx, self._ptr(D), ldd,
                                        self._ptr(cs), self._ptr(rs), self._stream()))
        return out

    def rmatmat(self, Y, colscale=None, rowscale=None, out=None):
        """X = diag(colscale) G^T diag(rowscale) Y; Y is (B, m), result (B, n)."""
        torch = _torch()
        Y, ldy = self._block(Y, self.m, "Y")
        B = Y.shape[0]
        if out is None:
            out = torch.empty((B, self.n), device=self.device, dtype=self.dtype)
        X, ldx = self._block(out, self.n, "out")
        cs = self._vec(colscale, self.n, "colscale")
        rs = self._vec(rowscale, self.m, "rowscale")
        _lib.check(_lib.lib().tf_rmatmat(self._h, B, self._ptr(Y), ldy, self._ptr(X), ldx,
                                         self._ptr(cs), self._ptr(rs), self._stream()))
        return out

    def matvec(self, x, colscale=None, rowscale=None, out=None):
        torch = _torch()
        x = self._vec(x, self.n, "x")
        if out is None:
            out = torch.empty(self.m, device=self.device, dtype=self.dtype)
        d = self._vec(out, self.m, "out")
        cs = self._vec(colscale, self.n, "colscale")
        rs = self._vec(rowscale, self.m, "rowscale")
        _lib.check(_lib.lib().tf_matvec(self._h, self._ptr(x), self._ptr(d), self._ptr(cs),
                                        self._ptr(rs), self._stream()))
        return out

    def rmatvec(self, y, colscale=None, rowscale=None, out=None):
        torch = _torch()
        y = self._vec(y, self.m, "y")
        if out is None:
            out = torch.empty(self.n, device=self.device, dtype=self.dtype)
        x = self._vec(out, self.n, "out")
        cs = self._vec(colscale, self.n, "colscale")
        rs = self._vec(rowscale, self.m, "rowscale")
        _lib.check(_lib.lib().tf_rmatvec(self._h, self._ptr(y), self._ptr(x), self._ptr(cs),
                                         self._ptr(rs), self._stream()))
        return out

    # -- host buffers: copies overlapped with the products (tf_products_host) -----------
    def _host_block(self, t, rows, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or t.device.type != "cpu" or t.dtype != self.dtype:
            raise TypeError(f"{name} must be a {self.dtype} host tensor")
        if t.dim() == 1:
            t = t.view(1, -1)
        if t.dim() != 2 or t.shape[1] != rows or t.stride(1) != 1 or (
                t.shape[0] > 1 and t.stride(0) < rows):
            raise ValueError(f"{name} must have shape (B, {rows}) with unit inner stride")
        return t, (t.stride(0) if t.shape[0] > 1 else rows)

    def products_host(self, X_host=None, Y_host=None, D_host=None, XT_host=None, chunks: int = 8,
                      colscale=None, rowscale=None):
        """G X and G^T Y for host blocks X (B1 x n) and Y (B2 x m) into host blocks
        D (B1 x m) and XT (B2 x n) (allocated pinned when not given); returns (D, XT).

        One tf_products_host call: the columns go through the device in `chunks` chunks
        whose copies in, products and copies out overlap (G^T's chunks ahead of G's, so
        that the two large copies use both directions of the host link).  Ordered on the
        current stream; synchronise it before reading the results.  Pass pinned tensors
        for overlapped copies."""
        torch = _torch()
        if X_host is None:
            X_host = torch.empty((0, self.n), dtype=self.dtype)
        if Y_host is None:
            Y_host = torch.empty((0, self.m), dtype=self.dtype)
        X, ldx = self._host_block(X_host, self.n, "X")
        Y, ldy = self._host_block(Y_host, self.m, "Y")
        B1, B2 = X.shape[0], Y.shape[0]
        if D_host is None:
            D_host = torch.empty((B1, self.m), dtype=self.dtype, pin_memory=B1 > 0)
        if XT_host is None:
            XT_host = torch.empty((B2, self.n), dtype=self.dtype, pin_memory=B2 > 0)
        D, ldd = self._host_block(D_host, self.m, "D")
        XT, ldxt = self._host_block(XT_host, self.n, "XT")
        if D.shape[0] != B1 or XT.shape[0] != B2:
            raise ValueError("output blocks must have as many columns as the inputs")
        cs = self._vec(colscale, self.n, "colscale")
        rs = self._vec(rowscale, self.m, "rowscale")
        p = lambda t: ctypes.c_void_p(t.data_ptr() if t.numel() else 0)
        _lib.check(_lib.lib().tf_products_host(
            self._h, B1, p(X), ldx, p(D), ldd, B2, p(Y), ldy, p(XT), ldxt, self._ptr(cs),
            self._ptr(rs), int(chunks), self._stream()))
        return D_host, XT_host

    def matmat_host(self, X_host, out_host=None, chunks: int = 4):
        """G X for a host block X (B x n) into host memory (B x m)."""
        return self.products_host(X_host, None, out_host, None, chunks)[0]

    def rmatmat_host(self, Y_host, out_host=None, chunks: int = 4):
        """G^T Y for a host block Y (B x m) into host memory (B x n)."""
        return self.products_host(None, Y_host, None, out_host, chunks)[1]

    # -- introspection ------------------------------------------------------------------
    def spectra(self):
        """Layer spectra (nz, n2, n1//2+1) complex, divided by n1*n2 (set-up output)."""
        torch = _torch()
        nh = self.n1 // 2 + 1
        cdt = torch.complex64 if self.dtype == torch.float32 else torch.complex128
        out = torch.empty((self.nz, self.n2, nh), dtype=cdt, device=self.device)
        nbytes = out.numel() * out.element_size()
        _lib.check(_lib.lib().tf_get_spectra(self._h, self._ptr(out), nbytes, self._stream()))
        return out

    def set_tuning(self, rows_tile=0, cols_tile=0, chunk_cols=0):
        _lib.check(_lib.lib().tf_set_tuning(self._h, rows_tile, cols_tile, chunk_cols))

    def tuning(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _lib.check(_lib.lib().tf_get_tuning(self._h, ctypes.byref(a), ctypes.byref(b),
                                            ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_radices(self, axis: int, radices):
        """Radix order of the generic engine's plan along x (axis 0) or y (axis 1)."""
        r = list(radices)
        arr = (ctypes.c_int * len(r))(*r)
        _lib.check(_lib.lib().tf_set_radices(self._h, int(axis), arr, len(r)))

    def radices(self, axis: int):
        arr = (ctypes.c_int * 16)()
        n = ctypes.c_int()
        _lib.check(_lib.lib().tf_get_radices(self._h, int(axis), arr, ctypes.byref(n)))
        return tuple(arr[:n.value])

    def set_engine(self, engine: int):
        """0: compile-time FFT plans where available (default); 1: generic engine."""
        _lib.check(_lib.lib().tf_set_engine(self._h, int(engine)))

    def engine(self):
        e, r, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(_lib.lib().tf_get_engine(self._h, ctypes.byref(e), ctypes.byref(r),
                                            ctypes.byref(c)))
        return e.value, bool(r.value), bool(c.value)

    def profile(self, enable: bool):
        _lib.check(_lib.lib().tf_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self):
        ms = (ctypes.c_double * 6)()
        la = (ctypes.c_int64 * 6)()
        co = (ctypes.c_int64 * 6)()
        _lib.check(_lib.lib().tf_profile_read(self._h, ms, la, co))
        return {STAGES[i]: (ms[i], la[i], co[i]) for i in range(6)}
