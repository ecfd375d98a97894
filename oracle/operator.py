"""Sensitivity matrix G and its products, FP64 (Sec. 2.1 Eq. (3); Sec. 2.5 Eq. (10); App. A).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.

Three routes to the same numbers:

* ``dense_G``: every entry G[(i,j),(p,q,r)] evaluated directly from the prism corner
  coordinates of station (i,j) and cell (p,q,r) (Sec. 2.1, Fig. 1), with no use of
  the BTTB structure.  Small grids only.
* ``fft_matvec`` / ``fft_rmatvec``: the paper's route (App. A): the first column of
  the BCCB extension of each layer block, reshaped to a (sx+nx-1) x (sy+ny-1) array T
  (``layer_tables``), is transformed with a 2-D FFT; ``G x = sum_r extract(ifft2(
  fft2(T_r) .* fft2(W_r)))`` with W_r the zero-embedded layer of x, and
  ``G^T y`` per layer with the conjugate spectrum (correlation), no layer sum.
* ``station_row``: one row of G by direct summation over all cells (O(n)), for
  sampled outputs at sizes where dense G does not fit.

Layout reading (the paper gives only the sizes of T and W, App. A): 0-based,
``T_r[s, t] = kernel at station-minus-cell-centre offset ((s-(nx-1)+pxl) dx,
(t-(ny-1)+pyl) dy)``; x is embedded at [0,nx) x [0,ny); d is read at
[nx-1, nx-1+sx) x [ny-1, ny-1+sy).  Any FFT size >= (sx+nx-1, sy+ny-1) with T zero
beyond gives the exact product.  Model index ``p + nx*(q + ny*r)``, data index
``i + sx*j``.
"""
from __future__ import annotations

import numpy as np

from . import prism

__all__ = ["layer_tables", "dense_G", "fft_matvec", "fft_rmatvec", "station_row",
           "kernel_eval"]


def kernel_eval(kind: str, x1, x2, y1, y2, z1, z2, inc=90.0, dec=0.0):
    """Entry of G for a prism with the given corner offsets (cell minus station)."""
    if kind == "gravity":
        return prism.gravity_cell(x1, x2, y1, y2, z1, z2)
    if kind == "magnetic":
        return prism.magnetic_cell(x1, x2, y1, y2, z1, z2, inc, dec)
    raise ValueError(kind)


def _layer_z(g, r):
    return g.z_edges[r] - g.station_z, g.z_edges[r + 1] - g.station_z


def layer_tables(g, kind: str, inc=90.0, dec=0.0) -> np.ndarray:
    """T_r arrays, shape (nz, sy+ny-1, sx+nx-1) indexed [r, t, s] (x fastest)."""
    s = np.arange(g.n1min, dtype=np.float64)
    t = np.arange(g.n2min, dtype=np.float64)
    # station minus cell centre; cell corners relative to the station follow
    ox = (s - (g.nx - 1) + g.pxl) * g.dx
    oy = (t - (g.ny - 1) + g.pyl) * g.dy
    cx = -ox[None, :]
    cy = -oy[:, None]
    out = np.empty((g.nz, g.n2min, g.n1min))
    for r in range(g.nz):
        z1, z2 = _layer_z(g, r)
        out[r] = kernel_eval(kind, cx - g.dx / 2, cx + g.dx / 2, cy - g.dy / 2,
                             cy + g.dy / 2, z1, z2, inc, dec)
    return out


def dense_G(g, kind: str, inc=90.0, dec=0.0) -> np.ndarray:
    """Dense m x n G from station and prism coordinates (no structure used)."""
    i = np.arange(g.sx)
    j = np.arange(g.sy)
    a = (i + g.pxl + 0.5) * g.dx                      # station x
    b = (j + g.pyl + 0.5) * g.dy                      # station y
    p = np.arange(g.nx)
    q = np.arange(g.ny)
    # station rows ordered i + sx*j, cell columns ordered p + nx*q (per layer)
    sa = np.tile(a, g.sy)[:, None]
    sb = np.repeat(b, g.sx)[:, None]
    cx0 = np.tile(p * g.dx, g.ny)[None, :]
    cy0 = np.repeat(q * g.dy, g.nx)[None, :]
    G = np.empty((g.m, g.n))
    nr = g.nx * g.ny
    for r in range(g.nz):
        z1, z2 = _layer_z(g, r)
        G[:, r * nr:(r + 1) * nr] = kernel_eval(
            kind, cx0 - sa, cx0 + g.dx - sa, cy0 - sb, cy0 + g.dy - sb, z1, z2, inc, dec)
    return G


def _fft_shape(g, n1=None, n2=None):
    n1 = g.n1min if n1 is None else n1
    n2 = g.n2min if n2 is None else n2
    if n1 < g.n1min or n2 < g.n2min:
        raise ValueError("FFT size below sx+nx-1 / sy+ny-1 wraps the convolution")
    return n2, n1          # numpy arrays are [y, x]


def fft_matvec(g, tables: np.ndarray, x: np.ndarray, n1=None, n2=None) -> np.ndarray:
    """d = G x by the BCCB embedding and 2-D FFTs, summed over layers (App. A)."""
    shape = _fft_shape(g, n1, n2)
    x3 = np.asarray(x, np.float64).reshape(g.nz, g.ny, g.nx)
    acc = np.zeros(shape, np.complex128)
    for r in range(g.nz):
        T = np.zeros(shape)
        T[:g.n2min, :g.n1min] = tables[r]
        W = np.zeros(shape)
        W[:g.ny, :g.nx] = x3[r]
        acc += np.fft.fft2(T) * np.fft.fft2(W)
    full = np.real(np.fft.ifft2(acc))
    d = full[g.ny - 1:g.ny - 1 + g.sy, g.nx - 1:g.nx - 1 + g.sx]
    return d.reshape(-1).copy()


def fft_rmatvec(g, tables: np.ndarray, y: np.ndarray, n1=None, n2=None) -> np.ndarray:
    """x = G^T y: per layer, extract(ifft2(conj(fft2(T_r)) .* fft2(Y))) (App. A)."""
    shape = _fft_shape(g, n1, n2)
    Y = np.zeros(shape)
    Y[g.ny - 1:g.ny - 1 + g.sy, g.nx - 1:g.nx - 1 + g.sx] = np.asarray(
        y, np.float64).reshape(g.sy, g.sx)
    Yh = np.fft.fft2(Y)
    out = np.empty((g.nz, g.ny, g.nx))
    for r in range(g.nz):
        T = np.zeros(shape)
        T[:g.n2min, :g.n1min] = tables[r]
        out[r] = np.real(np.fft.ifft2(np.conj(np.fft.fft2(T)) * Yh))[:g.ny, :g.nx]
    return out.reshape(-1)


def station_row(g, kind: str, i: int, j: int, inc=90.0, dec=0.0) -> np.ndarray:
    """Row (i + sx*j) of G by direct evaluation over all n cells."""
    a = (i + g.pxl + 0.5) * g.dx
    b = (j + g.pyl + 0.5) * g.dy
    cx0 = np.tile(np.arange(g.nx) * g.dx, g.ny)
    cy0 = np.repeat(np.arange(g.ny) * g.dy, g.nx)
    row = np.empty(g.n)
    nr = g.nx * g.ny
    for r in range(g.nz):
        z1, z2 = _layer_z(g, r)
        row[r * nr:(r + 1) * nr] = kernel_eval(
            kind, cx0 - a, cx0 + g.dx - a, cy0 - b, cy0 + g.dy - b, z1, z2, inc, dec)
    return row
