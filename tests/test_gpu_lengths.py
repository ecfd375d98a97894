"""Parity with the FP64 oracle at the transform lengths the large configurations run.

The small cases of test_gpu_products stay at FFT lengths <= 224.  Here the embeddings
(sx+nx-1) x (sy+ny-1) land in every length class of the compiled menus above that --
(224, 256], (256, 320], (320, 448], (448, 512] and the near-minimum lengths -- along both
axes, with and without the zero-upper-half first pass, FP32 and FP64, both FFT engines;
then the real c3 and c4 geometries (the benchmark's) on sampled columns.  The reference
is the oracle's FFT route (App. A; pinned to dense G on the CPU) per column, plus direct
row sums over all cells (Sec. 2.1) for sampled stations.

Tolerances (relative 2-norm per column): FP64 1e-12, FP32 2e-5.
"""
import numpy as np
import pytest

import synth
from oracle import operator as oop

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-12}

# name, grid, kind, inc, dec
LENGTHS = [
    # rows 229 (no zero-upper-half: nx = 130 > n1/2), cols 319 (ny = 220 > n2/2)
    ("r229_c319_full", synth.Grid(100, 100, 2, 15, 15, 60, 60), "gravity", 90.0, 0.0),
    # rows 369 (zero upper half), cols 489
    ("r369_c489", synth.Grid(180, 240, 2, 5, 5, 5, 5), "magnetic", 55.0, 12.0),
    # rows 487, cols 231
    ("r487_c231", synth.Grid(240, 110, 3, 4, 4, 6, 6), "gravity", 90.0, 0.0),
    # rows 299, cols 349
    ("r299_c349", synth.Grid(140, 170, 2, 10, 10, 5, 5), "magnetic", 35.0, -20.0),
    # rows 399, cols 499 (c4's two minimum lengths, swapped axes)
    ("r399_c499", synth.Grid(200, 250, 2), "gravity", 90.0, 0.0),
    # rows 303 (n1 = 320) with an odd row length (nx = 153) and ragged row counts (303 model
    # rows, 101 data rows): their last 16-row tiles are not whole 16-byte blocks, so the
    # row stages take the per-tile kernels instead of the bulk-copy ones
    ("r303_c201_odd", synth.Grid(151, 101, 3, 1, 1, 0, 0), "magnetic", 60.0, 5.0),
    # cols 257 (n2 = 320) with an odd layer row count (ny = 139): the forward column
    # kernel's second model column's layer tile must still start on a 128-byte boundary
    ("r79_c257_oddny", synth.Grid(37, 119, 3, 3, 3, 10, 10), "magnetic", 45.0, 10.0),
    # rows 261 (n1 = 320) with odd ny (117) and 351 model rows (a 7-row last tile)
    ("r261_c225_oddny", synth.Grid(126, 109, 3, 5, 5, 4, 4), "gravity", 90.0, 0.0),
]

_tables = {}


def tables(name, g, kind, inc, dec):
    if name not in _tables:
        _tables[name] = oop.layer_tables(g, kind, inc, dec)
    return _tables[name]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _dt(dtn):
    import torch
    return torch.float32 if dtn == "f32" else torch.float64


def _check_block(op, g, kind, inc, dec, T, dtn, B, seed, sample_cols, station_rows):
    import torch
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, g.n))
    Y = rng.standard_normal((B, g.m))
    cs = rng.uniform(0.5, 2.0, g.n)
    rs = rng.uniform(0.5, 2.0, g.m)
    t = lambda a: torch.tensor(a, dtype=_dt(dtn), device="cuda")
    D = op.matmat(t(X), colscale=t(cs), rowscale=t(rs)).double().cpu().numpy()
    Xt = op.rmatmat(t(Y), colscale=t(cs), rowscale=t(rs)).double().cpu().numpy()
    worst = 0.0
    for b in sample_cols:
        e1 = rel(D[b], rs * oop.fft_matvec(g, T, cs * X[b]))
        e2 = rel(Xt[b], cs * oop.fft_rmatvec(g, T, rs * Y[b]))
        worst = max(worst, e1, e2)
        assert e1 <= TOL[dtn], (b, e1)
        assert e2 <= TOL[dtn], (b, e2)
    for _ in range(station_rows):
        i, j = int(rng.integers(g.sx)), int(rng.integers(g.sy))
        b = int(rng.integers(B))
        row = oop.station_row(g, kind, i, j, inc, dec)
        ref = rs[i + g.sx * j] * (row @ (cs * X[b]))
        assert abs(D[b, i + g.sx * j] - ref) <= TOL[dtn] * np.abs(D[b]).max()
    return worst


@pytest.mark.parametrize("engine", [0, 1], ids=["compiled", "generic"])
@pytest.mark.parametrize("dtn", ["f64", "f32"])
@pytest.mark.parametrize("case", LENGTHS, ids=[c[0] for c in LENGTHS])
def test_large_lengths_match_oracle(case, dtn, engine):
    from paper_2004_13904_gb300 import Operator
    name, g, kind, inc, dec = case
    op = Operator(g, kind, inc, dec, dtype=_dt(dtn))
    op.set_engine(engine)
    assert op.n1 >= g.n1min and op.n2 >= g.n2min
    if engine == 0:
        assert op.engine() == (0, True, True), (op.n1, op.n2)   # both lengths compiled
    worst = _check_block(op, g, kind, inc, dec, tables(name, g, kind, inc, dec), dtn,
                         B=3, seed=5, sample_cols=range(3), station_rows=3)
    print(f"{name} {dtn} engine {engine}: fft {op.n1} x {op.n2}, worst rel err {worst:.2e}")
    op.close()


CONFIG_CASES = [("c3", "magnetic", 50.0, 10.0), ("c4", "gravity", 90.0, 0.0)]


@pytest.mark.parametrize("dtn", ["f64", "f32"])
@pytest.mark.parametrize("cfg", CONFIG_CASES, ids=[c[0] for c in CONFIG_CASES])
def test_config_geometries_sampled(cfg, dtn):
    """c3 (150 x 150 x 20) and c4 (250 x 200 x 20, the benchmark's workload) through the
    default engine: a 6-column block, 3 columns against the oracle's FFT route, 4 sampled
    stations against direct row sums."""
    from paper_2004_13904_gb300 import Operator
    name, kind, inc, dec = cfg
    g = synth.config_grid(name)
    op = Operator(g, kind, inc, dec, dtype=_dt(dtn))
    assert op.engine() == (0, True, True), (op.n1, op.n2)
    worst = _check_block(op, g, kind, inc, dec, tables(name, g, kind, inc, dec), dtn,
                         B=6, seed=9, sample_cols=(0, 3, 5), station_rows=4)
    print(f"{name} {dtn}: fft {op.n1} x {op.n2}, worst rel err {worst:.2e}")
    op.close()
