"""Autograd pair: back-propagated misfit gradients against the dense FP64 oracle and
against finite differences (FP64 and FP32)."""
import numpy as np
import pytest

import synth
from oracle import operator as oop

pytestmark = pytest.mark.gpu


def _setup(g, kind, inc, dec, dt):
    import torch
    from paper_2004_13904_gb300 import Operator
    return Operator(g, kind, inc, dec, dtype=dt)


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_misfit_gradient_matches_dense(dtn):
    import torch
    from paper_2004_13904_gb300.autograd import g_matmat
    dt = torch.float64 if dtn == "f64" else torch.float32
    g = synth.Grid(9, 7, 3, 1, 2, 2, 1)
    G = oop.dense_G(g, "magnetic", 50.0, 10.0)
    op = _setup(g, "magnetic", 50.0, 10.0, dt)
    rng = np.random.default_rng(4)
    m = rng.uniform(0, 0.1, g.n)
    d = G @ rng.uniform(0, 0.1, g.n)
    wd = 1.0 / (0.01 * np.abs(d) + 0.001 * np.abs(d).max())
    cs = rng.uniform(0.5, 2.0, g.n)
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    mt = t(m).requires_grad_(True)
    cst = t(cs).requires_grad_(True)
    r = g_matmat(op, mt, colscale=cst, rowscale=t(wd)) - t(wd * d)
    loss = 0.5 * (r * r).sum()
    loss.backward()
    res = wd * (G @ (cs * m) - d)
    ref_m = cs * (G.T @ (wd * res))
    ref_c = m * (G.T @ (wd * res))
    tol = 1e-12 if dtn == "f64" else 1e-4
    for got, ref in ((mt.grad, ref_m), (cst.grad, ref_c)):
        got = got.detach().cpu().numpy()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_finite_difference_directions_c3(dtn):
    """Directional derivatives of the weighted misfit on 64 random directions at the
    c3 magnetic size (150x150 stations, 150x150x20 cells)."""
    import torch
    from paper_2004_13904_gb300.autograd import g_matmat
    dt = torch.float64 if dtn == "f64" else torch.float32
    g = synth.config_grid("c3")
    op = _setup(g, "magnetic", 50.0, 10.0, dt)
    gen = torch.Generator(device="cuda").manual_seed(3)
    m = (0.1 * torch.rand(g.n, generator=gen, device="cuda", dtype=torch.float64)).to(dt)
    d = g_matmat(op, (0.1 * torch.rand(g.n, generator=gen, device="cuda",
                                       dtype=torch.float64)).to(dt)).detach()
    wd = 1.0 / (0.01 * d.abs() + 0.001 * d.abs().max())

    def f(x):
        r = wd * (g_matmat(op, x) - d)
        return 0.5 * (r.double() * r.double()).sum()

    x = m.clone().requires_grad_(True)
    f(x).backward()
    grad = x.grad.double()
    V = torch.randn(64, g.n, generator=gen, device="cuda", dtype=torch.float64)
    V /= V.norm(dim=1, keepdim=True)
    h = 1e-3 if dtn == "f64" else 3e-2
    errs = []
    with torch.no_grad():
        for v in V:
            # the misfit is quadratic, so the central difference is exact up to rounding
            fd = (f(m + (h * v).to(dt)) - f(m - (h * v).to(dt))) / (2 * h)
            an = (grad * v).sum()
            errs.append(float(abs(fd - an) / (abs(an) + 1e-30 * grad.norm())))
    errs = np.array(errs)
    assert np.median(errs) < (1e-9 if dtn == "f64" else 2e-2), np.median(errs)


def test_transpose_function_gradients():
    import torch
    from paper_2004_13904_gb300.autograd import g_rmatmat
    g = synth.Grid(6, 5, 2, 1, 1, 0, 2)
    G = oop.dense_G(g, "gravity")
    op = _setup(g, "gravity", 90.0, 0.0, torch.float64)
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((3, g.m))
    W = rng.standard_normal((3, g.n))
    cs = rng.uniform(0.5, 2, g.n)
    rs = rng.uniform(0.5, 2, g.m)
    t = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").requires_grad_(True)
    Yt, ct, rt = t(Y), t(cs), t(rs)
    loss = (g_rmatmat(op, Yt, colscale=ct, rowscale=rt) * torch.tensor(W, device="cuda")).sum()
    loss.backward()
    # loss = sum_b W_b . (c * G^T (r * Y_b))
    ref_Y = rs * (G @ (cs * W).T).T
    ref_c = (W * (G.T @ (rs * Y).T).T).sum(0)
    ref_r = (Y * (G @ (cs * W).T).T).sum(0)
    for got, ref in ((Yt.grad, ref_Y), (ct.grad, ref_c), (rt.grad, ref_r)):
        assert np.linalg.norm(got.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
