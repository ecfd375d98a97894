"""Pins of the oracle's IRLS solvers against textbook results on small dense problems."""
import math

import numpy as np
import pytest

import synth
from oracle import irls
from oracle import operator as oop


def _problem(seed=0, g=None, kind="gravity"):
    g = g or synth.Grid(7, 6, 3, 1, 1, 1, 1)
    G = oop.dense_G(g, kind, 50.0, 10.0)
    rng = np.random.default_rng(seed)
    wz = irls.depth_weights(g.z_edges, g.station_z, g.ny, g.nx, 0.8)
    wl = rng.uniform(0.5, 2.0, g.n)
    winv = 1.0 / (wz * wl)
    sigma = rng.uniform(0.5, 1.5, g.m) * 1e-3
    wd = 1.0 / sigma
    Gt = (wd[:, None] * G) * winv[None, :]
    rt = wd * (G @ rng.uniform(0, 1, g.n) * 0.1 + rng.standard_normal(g.m) * sigma)
    return g, G, Gt, rt, winv, wd


def test_gkb_factorisation_invariants():
    g, G, Gt, rt, _, _ = _problem()
    tp = 20
    f = irls.gkb(lambda x: Gt @ x, lambda y: Gt.T @ y, rt, tp, g.n)
    assert np.linalg.norm(f.A.T @ f.A - np.eye(tp)) < 1e-12
    assert np.linalg.norm(f.H.T @ f.H - np.eye(tp + 1)) < 1e-12
    assert np.linalg.norm(Gt @ f.A - f.H @ f.B) < 1e-12 * np.linalg.norm(Gt)
    # B is lower bidiagonal and H e_1 = r~ / ||r~||
    assert np.allclose(np.tril(np.triu(f.B, -1)), f.B)
    assert np.allclose(f.H[:, 0] * f.rnorm, rt)


def test_gkb_full_space_equals_tikhonov():
    g, G, Gt, rt, _, _ = _problem(1)
    m = g.m
    f = irls.gkb(lambda x: Gt @ x, lambda y: Gt.T @ y, rt, m, g.n)
    alpha = 0.3 * np.linalg.svd(Gt, compute_uv=False)[0]
    y, a, _ = irls.gkb_solution(f, m, alpha)
    direct = np.linalg.solve(Gt.T @ Gt + alpha ** 2 * np.eye(g.n), Gt.T @ rt)
    assert a == alpha
    assert np.linalg.norm(y - direct) < 1e-9 * np.linalg.norm(direct)


def test_rsvd_full_rank_singular_values_and_solution():
    g, G, Gt, rt, _, _ = _problem(2)
    m = g.m
    omega = synth.gaussian_columns(m, m, seed=9)
    f = irls.rsvd(lambda x: Gt @ x, lambda y: Gt.T @ y, omega)
    assert np.linalg.norm(f.Q.T @ f.Q - np.eye(m)) < 1e-12
    s_ref = np.linalg.svd(Gt, compute_uv=False)
    alpha = 0.1 * s_ref[0]
    y, a, St = irls.rsvd_solution(f, rt, m, alpha)
    assert np.allclose(St[:10], s_ref[:10], rtol=1e-10)
    direct = np.linalg.solve(Gt.T @ Gt + alpha ** 2 * np.eye(g.n), Gt.T @ rt)
    assert np.linalg.norm(y - direct) < 1e-8 * np.linalg.norm(direct)


def test_upre_matches_its_definition():
    # U(alpha) = ||G~ y_alpha - r~||^2 + 2 trace(influence) - m for whitened noise; for a
    # full-row-rank G~ the spectral form equals it exactly
    g, G, Gt, rt, _, _ = _problem(3)
    U, s, Vt = np.linalg.svd(Gt, full_matrices=False)
    beta = U.T @ rt
    for alpha in s[0] * np.array([1e-4, 1e-2, 0.3, 2.0]):
        y = np.linalg.solve(Gt.T @ Gt + alpha ** 2 * np.eye(g.n), Gt.T @ rt)
        infl = Gt @ np.linalg.solve(Gt.T @ Gt + alpha ** 2 * np.eye(g.n), Gt.T)
        direct = np.sum((Gt @ y - rt) ** 2) + 2 * np.trace(infl) - g.m
        assert abs(irls.upre(alpha, s, beta) - direct) <= 1e-8 * max(1.0, abs(direct))


def test_upre_minimiser_against_dense_search():
    rng = np.random.default_rng(5)
    s = np.sort(rng.uniform(1e-3, 10.0, 40))[::-1]
    beta = rng.standard_normal(40) * (1 + 20 * s)
    a = irls.upre_alpha(s, beta)
    dense = np.exp(np.linspace(math.log(s[-1] / 10), math.log(s[0]), 200001))
    vals = np.array([irls.upre(x, s, beta) for x in dense[::50]])
    best = dense[::50][int(np.argmin(vals))]
    assert irls.upre(a, s, beta) <= irls.upre(best, s, beta) + 1e-9
    assert abs(math.log(a / best)) < 0.01


def test_alpha_initial_closed_form():
    s = np.array([4.0, 2.0, 1.0, 1e-20])
    # mean over s > 0 (numerically: above 1e-14 s_1) is 7/3
    assert irls.alpha_initial(800, 100, s) == pytest.approx(8.0 ** 3.5 * 4.0 / (7.0 / 3.0))


def test_weights():
    wz = irls.depth_weights((0.0, 50.0, 150.0), 0.0, 2, 3, 1.4)
    assert wz.shape == (12,)
    assert wz[0] == pytest.approx(25.0 ** -1.4) and wz[-1] == pytest.approx(100.0 ** -1.4)
    wl = irls.focusing_weights(np.array([0.3, 0.0]), np.array([0.1, 0.0]), 1.0, 1e-9)
    assert wl[0] == pytest.approx((0.04 + 1e-9) ** -0.25)
    assert wl[1] == pytest.approx(1e-9 ** -0.25)


@pytest.mark.parametrize("solver", ["gkb", "rsvd"])
def test_irls_recovers_a_block_and_respects_bounds(solver):
    g = synth.Grid(12, 12, 4)
    G = oop.dense_G(g, "gravity")
    m_true = synth.block_model(g, 3, nbodies=1, lo=1.0, hi=1.0)
    d = G @ m_true
    sigma = 0.01 * np.abs(d) + 0.001 * np.abs(d).max()
    d_obs = d + sigma * synth.unit_noise(g.m, 3)
    wz = irls.depth_weights(g.z_edges, g.station_z, g.ny, g.nx, 0.8)
    # on 144 stations the spectrum decays slowly: the randomised range approximation
    # needs t close to m, while GKB succeeds with t = m/4
    t = g.m // 4 if solver == "gkb" else g.m - 10
    p = irls.IRLSParams(solver=solver, t=t, tp=(int(1.05 * t) if solver == "gkb" else t + 10),
                        kmax=15)
    omega = synth.gaussian_columns(g.m, p.tp, seed=11) if solver == "rsvd" else None
    m, rep = irls.irls(lambda x: G @ x, lambda y: G.T @ y, d_obs, sigma, g.n, wz, p, omega)
    assert m.min() >= 0.0 and m.max() <= 1.0
    re = np.linalg.norm(m - m_true) / np.linalg.norm(m_true)
    assert re < 0.2
    assert rep.chi2[-1] < rep.chi2[0]
    assert all(a > 0 for a in rep.alphas)

