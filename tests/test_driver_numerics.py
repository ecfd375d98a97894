"""Host numerics of the C IRLS drivers (no GPU): the tridiagonal eigen-iteration with
first eigenvector components, and the damped bidiagonal least squares solve, pinned to
numpy's dense routines on random and structured inputs."""
import ctypes

import numpy as np
import pytest

from paper_2004_13904_gb300 import _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def tridiag(d, e):
    d2, e2 = np.array(d, np.float64), np.zeros(len(d))
    e2[:len(e)] = e
    first = np.zeros(len(d))
    _lib.check(_lib.lib().tf_tridiag_eig_first(len(d), _dp(d2), _dp(e2), _dp(first)))
    return d2, first


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (60, 3), (301, 4)])
def test_tridiag_eigenvalues_and_first_components(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    w, Z = np.linalg.eigh(T)
    lam, first = tridiag(d, e)
    order = np.argsort(lam)
    assert np.allclose(lam[order], w, atol=1e-12 * max(1.0, abs(w).max()))
    # squared first components are the unique (sign-free) quantities
    assert np.allclose(first[order] ** 2, Z[0] ** 2, atol=1e-12)
    assert abs((first ** 2).sum() - 1.0) < 1e-12


def test_tridiag_gkb_shape_matches_singular_values():
    # B B^T of a lower bidiagonal (t_p+1) x t_p B: eigenvalues s_i^2 (and one zero),
    # first components = first row of U
    rng = np.random.default_rng(5)
    tp = 40
    gam = rng.uniform(0.1, 2.0, tp) * np.logspace(0, -6, tp)
    bet = rng.uniform(0.1, 2.0, tp) * np.logspace(0, -6, tp)
    B = np.zeros((tp + 1, tp))
    B[np.arange(tp), np.arange(tp)] = gam
    B[np.arange(tp) + 1, np.arange(tp)] = bet
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    dd = np.array([(gam[i] if i < tp else 0) ** 2 + (bet[i - 1] if i > 0 else 0) ** 2 for i in range(tp + 1)])
    ee = gam * bet
    lam, first = tridiag(dd, ee)
    order = np.argsort(-lam)[:tp]
    assert np.allclose(np.sqrt(np.maximum(lam[order], 0))[:10], s[:10], rtol=1e-12)
    assert np.allclose(first[order][:10] ** 2, U[0, :10] ** 2, atol=1e-12)


def test_tridiag_diagonal_and_repeated():
    lam, first = tridiag([3.0, 1.0, 2.0], [0.0, 0.0])
    assert sorted(lam) == [1.0, 2.0, 3.0]
    assert np.allclose(first ** 2, [1, 0, 0])
    lam, first = tridiag(np.full(5, 2.0), np.full(4, 1e-300))
    assert np.allclose(lam, 2.0)


@pytest.mark.parametrize("tp,alpha,seed", [(1, 0.3, 0), (5, 0.0, 1), (30, 1e-3, 2), (200, 0.5, 3)])
def test_damped_bidiagonal_solve(tp, alpha, seed):
    rng = np.random.default_rng(seed)
    gam = rng.uniform(0.2, 2.0, tp)
    bet = rng.uniform(0.2, 2.0, tp)
    b0 = 1.7
    B = np.zeros((tp + 1, tp))
    B[np.arange(tp), np.arange(tp)] = gam
    B[np.arange(tp) + 1, np.arange(tp)] = bet
    rhs = np.zeros(tp + 1)
    rhs[0] = b0
    A = np.vstack([B, alpha * np.eye(tp)])
    ref = np.linalg.lstsq(A, np.concatenate([rhs, np.zeros(tp)]), rcond=None)[0]
    # the Tikhonov-filtered SVD solution of Alg. 1 on all t_p terms is the same vector
    U, s, Vt = np.linalg.svd(B, full_matrices=False)
    svd_sol = Vt.T @ (s / (s * s + alpha * alpha) * (b0 * U[0]))
    y = np.zeros(tp)
    _lib.check(_lib.lib().tf_damped_bidiag_solve(tp, _dp(gam), _dp(bet), alpha, b0, _dp(y)))
    assert np.allclose(y, ref, rtol=1e-10, atol=1e-12)
    assert np.allclose(y, svd_sol, rtol=1e-10, atol=1e-12)


def test_helpers_reject_bad_arguments():
    L = _lib.lib()
    assert L.tf_damped_bidiag_solve(0, None, None, 1.0, 1.0, None) == _lib.TF_EINVAL
    assert L.tf_tridiag_eig_first(-1, None, None, None) == _lib.TF_EINVAL


def test_golub_kahan_route_keeps_small_singular_values():
    """The GKB driver's projected SVD: the Golub-Kahan tridiagonal of a realistic bidiagonal
    B (t_p = 1000, singular values graded over ten decades) gives every s_i to absolute
    accuracy ~eps s_1 and the first row of U to ~eps, against numpy's dense SVD.  The
    squared route through B B^T would lose the small s_i (error ~eps s_1^2 / s_i)."""
    rng = np.random.default_rng(17)
    tp = 1000
    grade = np.logspace(0, -10, tp)
    gam = rng.uniform(0.5, 1.5, tp) * grade
    bet = rng.uniform(0.5, 1.5, tp) * grade
    B = np.zeros((tp + 1, tp))
    B[np.arange(tp), np.arange(tp)] = gam
    B[np.arange(tp) + 1, np.arange(tp)] = bet
    U, s_ref, _ = np.linalg.svd(B, full_matrices=False)
    n = 2 * tp + 1
    e = np.zeros(n - 1)
    e[0::2] = gam
    e[1::2] = bet
    lam, first = tridiag(np.zeros(n), e)
    order = np.argsort(-lam)[:tp]
    s = lam[order]
    assert np.max(np.abs(s - s_ref)) <= 1e-13 * s_ref[0]
    # U(1, i)^2 = 2 first_i^2 where the singular values are well separated
    sep = np.r_[np.inf, np.diff(-s_ref)] > 1e-8 * s_ref[0]
    sep &= np.r_[np.diff(-s_ref), np.inf] > 1e-8 * s_ref[0]
    assert np.allclose(2 * first[order][sep] ** 2, U[0, sep] ** 2, atol=1e-12)
    # the B B^T route loses the small values to squaring
    dd = np.array([(gam[i] if i < tp else 0) ** 2 + (bet[i - 1] if i > 0 else 0) ** 2
                   for i in range(tp + 1)])
    lam2, _ = tridiag(dd, gam * bet)
    s2 = np.sqrt(np.maximum(np.sort(lam2)[::-1][:tp], 0))
    small = s_ref < 1e-6 * s_ref[0]
    assert np.max(np.abs(s2 - s_ref)[small] / s_ref[small]) > 1e-3
    assert np.max(np.abs(s - s_ref)[small] / s_ref[small]) < 1e-3
