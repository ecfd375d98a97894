"""Parity of the CUDA products with the FP64 oracle, through the C ABI.

Tolerances (relative 2-norm per column, against the oracle in FP64):
  FP64 path <= 1e-12, FP32 path <= 2e-5.
"""
import numpy as np
import pytest

import synth
from oracle import operator as oop

pytestmark = pytest.mark.gpu

TOL = {"f32": 2e-5, "f64": 1e-12}


def _torch():
    import torch
    return torch


def _dt(name):
    torch = _torch()
    return torch.float32 if name == "f32" else torch.float64


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SMALL = [
    ("grav_pad_asym", synth.Grid(5, 4, 3, 1, 2, 0, 1), "gravity", 90.0, 0.0),
    ("mag_aniso", synth.Grid(6, 7, 2, 2, 1, 1, 2, dx=40.0, dy=60.0, z_edges=(0.0, 30.0, 100.0)),
     "magnetic", 50.0, 10.0),
    ("mag_nz1", synth.Grid(8, 5, 1), "magnetic", 35.0, -20.0),
    ("single_cell", synth.Grid(1, 1, 1), "gravity", 90.0, 0.0),
    ("thin_strip", synth.Grid(1, 9, 2, 0, 0, 2, 3), "gravity", 90.0, 0.0),
    ("raised_stations", synth.Grid(4, 4, 2, station_z=-10.0), "gravity", 90.0, 0.0),
    ("c1_32x32x8", synth.config_grid("c1"), "gravity", 90.0, 0.0),
    ("ragged_37x23x5", synth.padded_grid(37, 23, 5, 0.08), "magnetic", 60.0, 15.0),
]

_cache = {}


class Ref:
    """Oracle products: dense G on tiny grids, else the oracle's FFT route (itself
    pinned to dense G on CPU), both FP64."""

    def __init__(self, g, kind, inc, dec):
        self.g = g
        if g.m * g.n <= 200000:
            self.G = oop.dense_G(g, kind, inc, dec)
            self.T = None
        else:
            self.G = None
            self.T = oop.layer_tables(g, kind, inc, dec)

    def mv(self, x):
        return self.G @ x if self.G is not None else oop.fft_matvec(self.g, self.T, x)

    def rmv(self, y):
        return self.G.T @ y if self.G is not None else oop.fft_rmatvec(self.g, self.T, y)


def ref(name, g, kind, inc, dec):
    if name not in _cache:
        _cache[name] = Ref(g, kind, inc, dec)
    return _cache[name]


def make_op(g, kind, inc, dec, dtn):
    from paper_2004_13904_gb300 import Operator
    return Operator(g, kind, inc, dec, dtype=_dt(dtn))


@pytest.mark.parametrize("engine", [0, 1], ids=["compiled", "generic"])
@pytest.mark.parametrize("dtn", ["f64", "f32"])
@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_products_match_dense(case, dtn, engine):
    torch = _torch()
    name, g, kind, inc, dec = case
    R = ref(name, g, kind, inc, dec)
    op = make_op(g, kind, inc, dec, dtn)
    op.set_engine(engine)
    assert op.engine()[0] == engine
    assert (op.m, op.n) == (g.m, g.n)
    rng = np.random.default_rng(1)
    B = 5
    X = rng.standard_normal((B, g.n))
    Y = rng.standard_normal((B, g.m))
    cs = rng.uniform(0.5, 2.0, g.n)
    rs = rng.uniform(0.5, 2.0, g.m)
    t = lambda a: torch.tensor(a, dtype=_dt(dtn), device="cuda")
    D = op.matmat(t(X)).cpu().numpy()
    Xt = op.rmatmat(t(Y)).cpu().numpy()
    Ds = op.matmat(t(X), colscale=t(cs), rowscale=t(rs)).cpu().numpy()
    Xs = op.rmatmat(t(Y), colscale=t(cs), rowscale=t(rs)).cpu().numpy()
    for b in range(B):
        assert rel(D[b], R.mv(X[b])) <= TOL[dtn]
        assert rel(Xt[b], R.rmv(Y[b])) <= TOL[dtn]
        assert rel(Ds[b], rs * R.mv(cs * X[b])) <= TOL[dtn]
        assert rel(Xs[b], cs * R.rmv(rs * Y[b])) <= TOL[dtn]
    d1 = op.matvec(t(X[0])).cpu().numpy()
    x1 = op.rmatvec(t(Y[0])).cpu().numpy()
    assert rel(d1, R.mv(X[0])) <= TOL[dtn]
    assert rel(x1, R.rmv(Y[0])) <= TOL[dtn]


@pytest.mark.parametrize("dtn", ["f64", "f32"])
@pytest.mark.parametrize("case", SMALL[:3] + SMALL[6:], ids=[c[0] for c in SMALL[:3] + SMALL[6:]])
def test_spectra_match_oracle(case, dtn):
    name, g, kind, inc, dec = case
    op = make_op(g, kind, inc, dec, dtn)
    T = oop.layer_tables(g, kind, inc, dec)
    ref = np.fft.rfft2(T, s=(op.n2, op.n1)) / (op.n1 * op.n2)
    got = op.spectra().cpu().numpy()
    assert got.shape == ref.shape
    assert rel(got, ref) <= (1e-13 if dtn == "f64" else 1e-6)


@pytest.mark.parametrize("tiles", [(4, 4), (8, 16), (16, 8)])
def test_tiles_and_ragged_chunks(tiles):
    torch = _torch()
    name, g, kind, inc, dec = SMALL[7]
    R = ref(name, g, kind, inc, dec)
    op = make_op(g, kind, inc, dec, "f64")
    op.set_engine(1)                            # tiles apply to the generic engine
    op.set_tuning(tiles[0], tiles[1], 3)        # chunks of 3 columns: 7 = 3 + 3 + 1
    assert op.tuning() == (tiles[0], tiles[1], 3)
    rng = np.random.default_rng(7)
    X = rng.standard_normal((7, g.n))
    Y = rng.standard_normal((7, g.m))
    D = op.matmat(torch.tensor(X, device="cuda")).cpu().numpy()
    Xt = op.rmatmat(torch.tensor(Y, device="cuda")).cpu().numpy()
    for b in range(7):
        assert rel(D[b], R.mv(X[b])) <= 1e-12
        assert rel(Xt[b], R.rmv(Y[b])) <= 1e-12


def test_strided_blocks_and_empty_block():
    torch = _torch()
    name, g, kind, inc, dec = SMALL[0]
    G = ref(name, g, kind, inc, dec).G
    op = make_op(g, kind, inc, dec, "f64")
    rng = np.random.default_rng(5)
    X = torch.tensor(rng.standard_normal((4, g.n + 7)), device="cuda")
    out = torch.full((4, g.m + 3), 123.0, dtype=torch.float64, device="cuda")
    op.matmat(X[:, :g.n], out=out[:, :g.m])
    o = out.cpu().numpy()
    assert rel(o[:, :g.m], X[:, :g.n].cpu().numpy() @ G.T) <= 1e-12
    assert np.all(o[:, g.m:] == 123.0)           # padding of the output block untouched
    empty = op.matmat(torch.empty((0, g.n), dtype=torch.float64, device="cuda"))
    assert empty.shape == (0, g.m)


def test_adjoint_identity_and_determinism_c3():
    torch = _torch()
    g = synth.config_grid("c3")
    op = make_op(g, "magnetic", 50.0, 10.0, "f64")
    rng = np.random.default_rng(9)
    x = torch.tensor(rng.standard_normal(g.n), device="cuda")
    y = torch.tensor(rng.standard_normal(g.m), device="cuda")
    gx = op.matvec(x)
    gty = op.rmatvec(y)
    lhs = float(gx @ y)
    rhs = float(x @ gty)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    assert torch.equal(op.matvec(x), gx)         # bitwise re-run equality


def test_compiled_plans_used_on_menu_sizes():
    op = make_op(synth.config_grid("c2"), "gravity", 90.0, 0.0, "f32")
    assert (op.n1, op.n2) == (224, 224)
    assert op.engine() == (0, True, True)
    op.set_engine(1)
    assert op.engine() == (1, False, False)


@pytest.mark.parametrize("dtn", ["f32", "f64"])
def test_c2_full_block_sampled(dtn):
    """The 1260-column c2 block the benchmark times, checked on sampled columns (FFT
    route of the oracle) and sampled outputs (direct row sums)."""
    torch = _torch()
    g = synth.config_grid("c2")
    op = make_op(g, "gravity", 90.0, 0.0, dtn)
    B = 1260
    X = synth.gaussian_columns(g.n, B, seed=123)
    Y = synth.gaussian_columns(g.m, B, seed=321)
    Xd = torch.tensor(X, dtype=_dt(dtn), device="cuda")
    Yd = torch.tensor(Y, dtype=_dt(dtn), device="cuda")
    D = op.matmat(Xd).cpu().numpy()
    Xt = op.rmatmat(Yd).cpu().numpy()
    T = oop.layer_tables(g, "gravity")
    for b in (0, 617, B - 1):
        assert rel(D[b], oop.fft_matvec(g, T, X[b])) <= TOL[dtn]
        assert rel(Xt[b], oop.fft_rmatvec(g, T, Y[b])) <= TOL[dtn]
    rng = np.random.default_rng(2)
    for _ in range(6):
        i, j = int(rng.integers(g.sx)), int(rng.integers(g.sy))
        row = oop.station_row(g, "gravity", i, j)
        b = int(rng.integers(B))
        ref = row @ X[b]
        scale = np.abs(D[b]).max()
        assert abs(D[b, i + g.sx * j] - ref) <= TOL[dtn] * scale


def test_errors_through_abi():
    import ctypes
    torch = _torch()
    from paper_2004_13904_gb300 import _lib
    g = SMALL[0][1]
    op = make_op(g, "gravity", 90.0, 0.0, "f32")
    L = _lib.lib()
    X = torch.zeros((2, g.n), device="cuda")
    D = torch.zeros((2, g.m), device="cuda")
    st = L.tf_matmat(op._h, 2, ctypes.c_void_p(X.data_ptr()), g.n - 1,
                     ctypes.c_void_p(D.data_ptr()), g.m, None, None, None)
    assert st == _lib.TF_EINVAL
    assert L.tf_matmat(op._h, -1, None, g.n, None, g.m, None, None, None) == _lib.TF_EINVAL
    assert L.tf_set_tuning(op._h, 3, 0, 0) == _lib.TF_EINVAL
    with pytest.raises(TypeError):
        op.matmat(torch.zeros((2, g.n), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        op.matvec(torch.zeros(g.n + 1, device="cuda"))


@pytest.mark.parametrize("chunks", [1, 3])
def test_host_pipeline_matches_device_products(chunks):
    torch = _torch()
    g = SMALL[7][1]
    op = make_op(g, "magnetic", 60.0, 15.0, "f32")
    rng = np.random.default_rng(12)
    X = torch.tensor(rng.standard_normal((11, g.n)), dtype=torch.float32).pin_memory()
    Y = torch.tensor(rng.standard_normal((11, g.m)), dtype=torch.float32).pin_memory()
    D = op.matmat_host(X, chunks=chunks)
    XT = op.rmatmat_host(Y, chunks=chunks)
    torch.cuda.synchronize()
    assert torch.equal(D, op.matmat(X.cuda()).cpu())
    assert torch.equal(XT, op.rmatmat(Y.cuda()).cpu())


@pytest.mark.gpu
@pytest.mark.parametrize("chunks", [1, 3, 20])
def test_products_host_matches_device_products(chunks):
    # both directions in one pipeline, blocks of different widths (and chunks > columns)
    torch = _torch()
    g = SMALL[7][1]
    op = make_op(g, "gravity", 90.0, 0.0, "f32")
    rng = np.random.default_rng(13)
    X = torch.tensor(rng.standard_normal((9, g.n)), dtype=torch.float32).pin_memory()
    Y = torch.tensor(rng.standard_normal((5, g.m)), dtype=torch.float32).pin_memory()
    for _ in range(2):
        D, XT = op.products_host(X, Y, chunks=chunks)
        torch.cuda.synchronize()
        assert torch.equal(D, op.matmat(X.cuda()).cpu())
        assert torch.equal(XT, op.rmatmat(Y.cuda()).cpu())
