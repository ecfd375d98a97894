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


TOL = {"f64": 1e-12, "f32": 2e-5}      # relative 2-norm tolerance of one product column


def _fd_check(f_dir, grad, grad_ref, V, h, eps):
    """Central differences of the quadratic misfit along each unit direction v, against
    the back-propagated gradient.  For a quadratic the central difference has no
    truncation error, so |fd - grad.v| is bounded by rounding alone:
      * each misfit value 0.5 ||r||^2 is computed from a residual r whose product part is
        within eps * P of exact (P = ||W_d G x||, the product tolerance per column), so
        it is off by at most eps ||r|| P + (eps P)^2 / 2, and the difference quotient by
        (e+ + e-) / (2 h);
      * grad.v differs from the exact directional derivative by at most
        ||grad - grad_ref|| (||v|| = 1), grad_ref being the FP64 oracle's gradient.
    Every direction must meet its own bound (worst case, not a median)."""
    worst, bounds, derivs = 0.0, 0.0, 0.0
    for v in V:
        (fp, rp, pp), (fm, rm, pm) = f_dir(v, h), f_dir(v, -h)
        fd = (fp - fm) / (2 * h)
        an = float(grad @ v)
        e_f = lambda r, p: eps * r * p + 0.5 * (eps * p) ** 2
        bound = (e_f(rp, pp) + e_f(rm, pm)) / (2 * h) + float(np.linalg.norm(grad - grad_ref))
        bound *= 1.0 + 1e-9
        worst = max(worst, abs(fd - an) / bound)
        bounds += bound
        derivs += abs(float(grad_ref @ v))
    assert worst <= 1.0, worst
    # the bounds are small against the derivatives themselves, so the check pins the
    # adjoint (a wrong transpose is off by about the derivative's own size)
    assert bounds < 0.1 * derivs, (bounds, derivs)
    return worst


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_finite_difference_directions_c3(dtn):
    """Directional derivatives of the weighted misfit 0.5 ||W_d (G m - d)||^2 on 64 random
    unit directions at the c3 magnetic size (150x150 stations, 150x150x20 cells), each
    within a worst-case rounding bound derived from the product tolerance and h; the
    back-propagated gradient itself against the FP64 oracle's G^T W_d^2 (G m - d)."""
    import torch
    from paper_2004_13904_gb300.autograd import g_matmat
    dt = torch.float64 if dtn == "f64" else torch.float32
    g = synth.config_grid("c3")
    T = oop.layer_tables(g, "magnetic", 50.0, 10.0)
    op = _setup(g, "magnetic", 50.0, 10.0, dt)
    rng = np.random.default_rng(3)
    m = 0.1 * rng.random(g.n)
    d = oop.fft_matvec(g, T, 0.1 * rng.random(g.n))
    wd = 1.0 / (0.01 * np.abs(d) + 0.001 * np.abs(d).max())
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    wdt, dwt = t(wd), t(wd * d)

    x = t(m).requires_grad_(True)
    r = g_matmat(op, x, rowscale=wdt) - dwt
    (0.5 * (r.double() * r.double()).sum()).backward()
    grad = x.grad.double().cpu().numpy()
    grad_ref = oop.fft_rmatvec(g, T, wd * wd * (oop.fft_matvec(g, T, m) - d))
    assert np.linalg.norm(grad - grad_ref) <= 4 * TOL[dtn] * np.linalg.norm(grad_ref)

    def f_dir(v, h):
        with torch.no_grad():
            xp = m + h * v
            gx = g_matmat(op, t(xp), rowscale=wdt)
            rr = (gx - dwt).double()
            return (0.5 * float((rr * rr).sum()), float(rr.norm()), float(gx.double().norm()))

    V = rng.standard_normal((64, g.n))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    worst = _fd_check(f_dir, grad, grad_ref, V, 10.0, TOL[dtn])
    print(f"c3 {dtn}: worst |fd - grad.v| / bound over 64 directions = {worst:.3f}")


@pytest.mark.parametrize("dtn", ["f64", "f32"])
def test_finite_difference_directions_dense(dtn):
    """The same worst-case finite-difference check on a grid small enough for the
    oracle's dense G, whose gradient G^T W_d^2 (G m - d) is the reference."""
    import torch
    from paper_2004_13904_gb300.autograd import g_matmat
    dt = torch.float64 if dtn == "f64" else torch.float32
    g = synth.Grid(11, 9, 4, 2, 1, 1, 2)
    G = oop.dense_G(g, "magnetic", 50.0, 10.0)
    op = _setup(g, "magnetic", 50.0, 10.0, dt)
    rng = np.random.default_rng(11)
    m = 0.1 * rng.random(g.n)
    d = G @ (0.1 * rng.random(g.n))
    wd = 1.0 / (0.01 * np.abs(d) + 0.001 * np.abs(d).max())
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda")
    wdt, dwt = t(wd), t(wd * d)
    x = t(m).requires_grad_(True)
    r = g_matmat(op, x, rowscale=wdt) - dwt
    (0.5 * (r.double() * r.double()).sum()).backward()
    grad = x.grad.double().cpu().numpy()
    grad_ref = G.T @ (wd * wd * (G @ m - d))
    assert np.linalg.norm(grad - grad_ref) <= 4 * TOL[dtn] * np.linalg.norm(grad_ref)

    def f_dir(v, h):
        with torch.no_grad():
            gx = g_matmat(op, t(m + h * v), rowscale=wdt)
            rr = (gx - dwt).double()
            return (0.5 * float((rr * rr).sum()), float(rr.norm()), float(gx.double().norm()))

    V = rng.standard_normal((32, g.n))
    V /= np.linalg.norm(V, axis=1, keepdims=True)
    _fd_check(f_dir, grad, grad_ref, V, 1.0, TOL[dtn])


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
