"""Host-side pieces of the GPU inversion drivers (no GPU needed): the projected-problem
decompositions and the regularisation-parameter choice, checked against dense LAPACK
and the definition of UPRE."""
import math

import numpy as np
import pytest


def test_large_bidiagonal_route_matches_dense_svd():
    # the GPU driver's tridiagonal route for large GKB bidiagonals (used above 512 terms)
    # gives the same regularised solution as a dense SVD
    pytest.importorskip("scipy")
    from paper_2004_13904_gb300.irls import bidiag_svd
    rng = np.random.default_rng(0)
    n = 700
    gam = np.sort(rng.uniform(1e-4, 10.0, n))[::-1]
    bet = rng.uniform(1e-4, 3.0, n)
    B = np.zeros((n + 1, n))
    B[np.arange(n), np.arange(n)] = gam
    B[np.arange(n) + 1, np.arange(n)] = bet
    U, s_ref, Vh_ref = np.linalg.svd(B, full_matrices=False)
    u1, s, Vh = bidiag_svd(B)
    assert np.max(np.abs(s - s_ref)) <= 1e-13 * s_ref[0]
    for alpha in (1e-2, 0.3, 3.0):
        y_ref = Vh_ref.T @ (U[0] * s_ref / (s_ref ** 2 + alpha ** 2))
        y = Vh.T @ (u1 * s / (s ** 2 + alpha ** 2))
        assert np.linalg.norm(y - y_ref) <= 1e-10 * np.linalg.norm(y_ref)


def test_choose_alpha_matches_dense_search():
    from paper_2004_13904_gb300.irls import choose_alpha, upre_value
    rng = np.random.default_rng(5)
    s = np.sort(rng.uniform(1e-3, 10.0, 40))[::-1]
    coef = rng.standard_normal(40) * (1 + 20 * s)
    a = choose_alpha(s, coef)
    dense = np.exp(np.linspace(math.log(s[-1] / 10), math.log(s[0]), 4001))
    vals = upre_value(dense, s, coef)
    best = dense[int(np.argmin(vals))]
    assert upre_value(a, s, coef) <= upre_value(best, s, coef) + 1e-9
    assert abs(math.log(a / best)) < 0.01


def test_upre_value_definition():
    from paper_2004_13904_gb300.irls import upre_value
    s = np.array([3.0, 1.0, 0.2])
    c = np.array([1.0, -2.0, 0.5])
    a = 0.7
    f = s ** 2 / (s ** 2 + a ** 2)
    assert upre_value(a, s, c) == pytest.approx(np.sum(((1 - f) * c) ** 2) + 2 * f.sum() - 3)
