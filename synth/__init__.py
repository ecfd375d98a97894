"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module holds geometry and random draws only: grid sizes, padding counts, seeded
model bodies, Gaussian columns and unit-variance noise draws.  It contains none of the
forward-modelling arithmetic (no prism kernels, no FFTs, no products), so the CPU oracle
and the CUDA path can both take their inputs from here without sharing any of the
method's code.

Geometry conventions (Sec. 2.1, Fig. 1; padding rule Sec. 3.2):
  * cells are cubes of side ``dx = dy`` (and ``z_edges`` in depth), indexed
    ``0 <= p < nx``, ``0 <= q < ny``, ``0 <= r < nz``; cell ``p`` spans ``[p dx, (p+1) dx]``;
  * stations sit at z = ``station_z`` over the centres of the unpadded surface cells:
    station ``i`` is over cell ``i + pxl``, i.e. at ``x = (i + pxl + 1/2) dx``;
  * the model vector is ordered ``p + nx*(q + ny*r)`` and the data vector ``i + sx*j``;
  * padding per side is ``round(pad * s)`` with MATLAB rounding (halves away from zero),
    which reproduces the padded sizes of the paper's Table 2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Grid", "round_half_away", "padded_grid", "config_grid", "CONFIGS",
    "block_model", "dike_model", "config_model", "gaussian_columns",
    "unit_noise", "batch_problems",
]


def round_half_away(v: float) -> int:
    """MATLAB-style rounding: halves go away from zero (Python's round() does not)."""
    return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)


@dataclasses.dataclass(frozen=True)
class Grid:
    """Station/volume geometry of one problem (Sec. 2.1, Fig. 1)."""
    sx: int
    sy: int
    nz: int
    pxl: int = 0
    pxr: int = 0
    pyl: int = 0
    pyr: int = 0
    dx: float = 50.0
    dy: float = 50.0
    z_edges: tuple = ()
    station_z: float = 0.0

    def __post_init__(self):
        if not self.z_edges:
            object.__setattr__(self, "z_edges", tuple(50.0 * k for k in range(self.nz + 1)))
        if len(self.z_edges) != self.nz + 1:
            raise ValueError("z_edges must have nz+1 entries")

    @property
    def nx(self) -> int:
        return self.sx + self.pxl + self.pxr

    @property
    def ny(self) -> int:
        return self.sy + self.pyl + self.pyr

    @property
    def m(self) -> int:
        return self.sx * self.sy

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n1min(self) -> int:
        return self.sx + self.nx - 1

    @property
    def n2min(self) -> int:
        return self.sy + self.ny - 1


def padded_grid(sx: int, sy: int, nz: int, pad: float = 0.0, dx: float = 50.0,
                dy: float = 50.0, dz: float = 50.0, station_z: float = 0.0) -> Grid:
    """Grid with ``round(pad*s)`` padding cells on each side (Sec. 3.2)."""
    px = round_half_away(pad * sx)
    py = round_half_away(pad * sy)
    return Grid(sx, sy, nz, px, px, py, py, dx, dy,
                tuple(dz * k for k in range(nz + 1)), station_z)


# The five workloads: station grid, depth layers and padding fraction.
CONFIGS = {
    "c1": dict(sx=32, sy=32, nz=8, pad=0.0, kind="gravity"),
    "c2": dict(sx=100, sy=100, nz=10, pad=0.05, kind="gravity"),
    "c3": dict(sx=150, sy=150, nz=20, pad=0.0, kind="magnetic", inc=50.0, dec=10.0),
    "c4": dict(sx=250, sy=200, nz=20, pad=0.0, kind="gravity"),
}


def config_grid(name: str) -> Grid:
    c = CONFIGS[name]
    return padded_grid(c["sx"], c["sy"], c["nz"], c["pad"])


def _box(model: np.ndarray, g: Grid, p0, p1, q0, q1, r0, r1, value: float) -> None:
    m3 = model.reshape(g.nz, g.ny, g.nx)
    m3[max(r0, 0):min(r1, g.nz), max(q0, 0):min(q1, g.ny), max(p0, 0):min(p1, g.nx)] = value


def block_model(g: Grid, seed: int, nbodies: int = 2, lo: float = 1.0,
                hi: float = 1.0) -> np.ndarray:
    """Zero model with ``nbodies`` seeded axis-aligned blocks of value in [lo, hi]."""
    rng = np.random.default_rng(seed)
    model = np.zeros(g.n)
    for _ in range(nbodies):
        wx = int(rng.integers(max(2, g.sx // 8), max(3, g.sx // 3)))
        wy = int(rng.integers(max(2, g.sy // 8), max(3, g.sy // 3)))
        wz = int(rng.integers(1, max(2, g.nz // 2)))
        p0 = g.pxl + int(rng.integers(0, max(1, g.sx - wx)))
        q0 = g.pyl + int(rng.integers(0, max(1, g.sy - wy)))
        r0 = int(rng.integers(0, max(1, g.nz - wz)))
        _box(model, g, p0, p0 + wx, q0, q0 + wy, r0, r0 + wz, float(rng.uniform(lo, hi)))
    return model


def dike_model(g: Grid, seed: int, value: float = 1.0, layers: int = 6) -> np.ndarray:
    """A dipping dike: a slab whose x-position shifts by one cell per layer."""
    rng = np.random.default_rng(seed)
    model = np.zeros(g.n)
    width = max(1, g.sx // 12)
    p0 = g.pxl + int(rng.integers(g.sx // 4, g.sx // 2))
    q0 = g.pyl + int(rng.integers(0, max(1, g.sy // 4)))
    q1 = q0 + max(2, g.sy // 2)
    r_start = int(rng.integers(0, max(1, g.nz - layers)))
    for k in range(min(layers, g.nz - r_start)):
        _box(model, g, p0 + k, p0 + k + width, q0, q1, r_start + k, r_start + k + 1, value)
    return model


def config_model(name: str, seed: int) -> np.ndarray:
    """The seeded true model of a named workload (values in the paper's ranges)."""
    g = config_grid(name)
    if name == "c1":
        return block_model(g, seed, nbodies=2, lo=1.0, hi=1.0)
    if name == "c2":
        return np.maximum(dike_model(g, seed, float(np.random.default_rng(seed).uniform(0.5, 1.0))),
                          block_model(g, seed + 100, nbodies=2, lo=0.3, hi=1.0))
    if name == "c3":
        return block_model(g, seed, nbodies=3, lo=0.02, hi=0.1)
    if name == "c4":
        return np.maximum(dike_model(g, seed), block_model(g, seed + 100, nbodies=5, lo=0.2, hi=1.0))
    raise KeyError(name)


def gaussian_columns(rows: int, cols: int, seed: int = 123) -> np.ndarray:
    """i.i.d. N(0,1) float64 matrix, column-major (shape (cols, rows): one column per row)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((cols, rows))


def unit_noise(m: int, seed: int) -> np.ndarray:
    """Unit-variance Gaussian draws e of the noise model (Sec. 3.1); callers scale them."""
    return np.random.default_rng(seed + 7919).standard_normal(m)


@dataclasses.dataclass(frozen=True)
class Problem:
    grid: Grid
    kind: str
    inc: float = 90.0
    dec: float = 0.0


def batch_problems(count: int = 64, seed: int = 5) -> List[Problem]:
    """Uneven batch: grids from 32x32x8 to 128x128x16, 0-10 % padding, half magnetic."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        sx = int(rng.integers(32, 129))
        sy = int(rng.integers(32, 129))
        nz = int(rng.integers(8, 17))
        pad = float(rng.uniform(0.0, 0.10))
        g = padded_grid(sx, sy, nz, pad)
        if k % 2 == 0:
            out.append(Problem(g, "gravity"))
        else:
            out.append(Problem(g, "magnetic", float(rng.uniform(30.0, 70.0)), 10.0))
    return out
