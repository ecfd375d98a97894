"""IRLS focusing inversion with the GKB and RSVD solvers, FP64 (Sec. 2.2-2.4, Alg. 1-2,
Sec. 3.1).

TEST INFRASTRUCTURE ONLY: part of the CPU oracle.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import it.

The algorithms follow the paper's steps in its order and notation:

* ``gkb``: Alg. 1, Golub-Kahan bidiagonalisation of G~ = W_d G W^-1 started from r~,
  with modified Gram-Schmidt against all earlier columns of A and H;
* ``gkb_solution``: SVD of the (t_p+1) x t_p bidiagonal B, truncated UPRE on t terms,
  y = ||r~|| A V Gamma(alpha, Sigma) U(1,:)^T with all t_p terms;
* ``rsvd``: Alg. 2, randomised SVD with one power iteration (Omega is an input);
* ``rsvd_solution``: eig of (B^T B + (B^T B)^T)/2, S = sqrt|D| sorted descending,
  t-term truncation, y = Q V~ Gamma U~^T (B^T r~);
* ``irls``: Sec. 2.3 with W = W_z W_L^(k), W_L^(1) = I,
  (W_L^(k))_ii = ((m^(k-1)_i - m^(k-2)_i)^2 + eps^2)^((lambda-2)/4),
  r~ = W_d (d_obs - G m^(k-1)), m^(k) = clip(m^(k-1) + W^-1 z, bounds),
  alpha^(1) from Eq. (11), UPRE for k > 1, stop on Eq. (12) or after K_max.

Readings (the paper is silent): UPRE is Vogel's unbiased predictive risk for whitened
noise on the t retained terms, U(alpha) = sum (alpha^2/(s^2+alpha^2))^2 beta^2
+ 2 sum s^2/(s^2+alpha^2) - t, minimised on 200 log-spaced points over
[max(s_t, 1e-14 s_1)/10, s_1] and refined by golden-section search between the grid
neighbours of the best point (smallest index wins ties); the mean in Eq. (11) runs over
the t retained singular values above 1e-14 s_1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

# ---------------------------------------------------------------------------------------
# weights


def depth_weights(z_edges, station_z: float, ny: int, nx: int, beta: float) -> np.ndarray:
    """Diagonal of W_z: per layer (mean depth)^(-beta), Sec. 2.2."""
    z = np.asarray(z_edges, np.float64) - station_z
    zbar = 0.5 * (z[:-1] + z[1:])
    return np.repeat(zbar ** (-beta), nx * ny)


def focusing_weights(m_prev, m_prev2, lam: float, eps2: float) -> np.ndarray:
    """Diagonal of W_L^(k) from the two previous iterates, Sec. 2.3."""
    return ((m_prev - m_prev2) ** 2 + eps2) ** ((lam - 2.0) / 4.0)


# ---------------------------------------------------------------------------------------
# regularisation parameter


def upre(alpha: float, s: np.ndarray, beta: np.ndarray) -> float:
    """t-term UPRE functional (whitened noise), up to an alpha-independent constant."""
    a2 = alpha * alpha
    f = s * s / (s * s + a2)
    return float(np.sum(((1.0 - f) * beta) ** 2) + 2.0 * np.sum(f) - s.size)


def upre_alpha(s: np.ndarray, beta: np.ndarray) -> float:
    """Minimiser of ``upre``: log grid of 200 points, then golden-section refinement."""
    s = np.asarray(s, np.float64)
    lo = max(s[-1], 1e-14 * s[0]) / 10.0
    hi = s[0]
    grid = np.exp(np.linspace(math.log(lo), math.log(hi), 200))
    vals = np.array([upre(a, s, beta) for a in grid])
    k = int(np.argmin(vals))
    a = math.log(grid[max(k - 1, 0)])
    b = math.log(grid[min(k + 1, grid.size - 1)])
    phi = (math.sqrt(5.0) - 1.0) / 2.0
    c = b - phi * (b - a)
    d = a + phi * (b - a)
    fc = upre(math.exp(c), s, beta)
    fd = upre(math.exp(d), s, beta)
    for _ in range(80):
        if fc <= fd:
            b, d, fd = d, c, fc
            c = b - phi * (b - a)
            fc = upre(math.exp(c), s, beta)
        else:
            a, c, fc = c, d, fd
            d = a + phi * (b - a)
            fd = upre(math.exp(d), s, beta)
    best = math.exp(0.5 * (a + b))
    return best if upre(best, s, beta) <= vals[k] else float(grid[k])


def alpha_initial(n: int, m: int, s: np.ndarray) -> float:
    """Eq. (11): (n/m)^3.5 * s_1 / mean(s_i > 0)."""
    s = np.asarray(s, np.float64)
    pos = s[s > 1e-14 * s[0]]
    return (n / m) ** 3.5 * s[0] / float(np.mean(pos))


def tikhonov_filter(alpha: float, s: np.ndarray) -> np.ndarray:
    """Gamma(alpha, Sigma) = diag(s / (s^2 + alpha^2))."""
    return s / (s * s + alpha * alpha)


# ---------------------------------------------------------------------------------------
# solvers


@dataclasses.dataclass
class GKBFactor:
    A: np.ndarray        # n x tp
    H: np.ndarray        # m x (tp+1)
    B: np.ndarray        # (tp+1) x tp, lower bidiagonal
    rnorm: float


def gkb(apply_Gt: Callable, apply_GtT: Callable, rt: np.ndarray, tp: int, n: int) -> GKBFactor:
    """Alg. 1: G~ A = H B with MGS re-orthogonalisation of A and H."""
    m = rt.size
    a = np.zeros(n)
    B = np.zeros((tp + 1, tp))
    H = np.zeros((m, tp + 1))
    A = np.zeros((n, tp))
    beta = float(np.linalg.norm(rt))
    h = rt / beta
    H[:, 0] = h
    rnorm = beta
    for i in range(tp):
        b = apply_GtT(h) - beta * a
        for j in range(i):
            b = b - (A[:, j] @ b) * A[:, j]
        gamma = float(np.linalg.norm(b))
        a = b / gamma
        B[i, i] = gamma
        A[:, i] = a
        c = apply_Gt(a) - gamma * h
        for j in range(i + 1):
            c = c - (H[:, j] @ c) * H[:, j]
        beta = float(np.linalg.norm(c))
        h = c / beta
        B[i + 1, i] = beta
        H[:, i + 1] = h
    return GKBFactor(A, H, B, rnorm)


def gkb_solution(f: GKBFactor, t: int, alpha: Optional[float] = None):
    """Alg. 1 final steps: SVD of B, truncated UPRE on t terms, y with all t_p terms.
    Returns (y, alpha, singular values of B)."""
    U, s, Vt = np.linalg.svd(f.B, full_matrices=False)
    coef = f.rnorm * U[0, :]
    if alpha is None:
        alpha = upre_alpha(s[:t], coef[:t])
    y = f.A @ (Vt.T @ (tikhonov_filter(alpha, s) * coef))
    return y, alpha, s


@dataclasses.dataclass
class RSVDFactor:
    Q: np.ndarray        # n x tp (the last QR factor)
    B: np.ndarray        # m x tp


def rsvd(apply_Gt: Callable, apply_GtT: Callable, omega: np.ndarray) -> RSVDFactor:
    """Alg. 2 up to B = G~ Q: one power iteration, omega is t_p x m Gaussian."""
    Y = np.stack([apply_GtT(w) for w in omega])                 # Omega G~, t_p x n
    Q, _ = np.linalg.qr(Y.T)                                      # n x t_p
    Y1 = np.stack([apply_Gt(q) for q in Q.T], axis=1)             # G~ Q, m x t_p
    Q1, _ = np.linalg.qr(Y1)                                      # m x t_p
    Y2 = np.stack([apply_GtT(q) for q in Q1.T])                   # Q1^T G~, t_p x n
    Q2, _ = np.linalg.qr(Y2.T)                                    # n x t_p
    B = np.stack([apply_Gt(q) for q in Q2.T], axis=1)             # G~ Q2, m x t_p
    return RSVDFactor(Q2, B)


def rsvd_solution(f: RSVDFactor, rt: np.ndarray, t: int, alpha: Optional[float] = None):
    """Alg. 2 final steps: eig of the symmetrised B^T B, t-term truncation, UPRE, y.
    Returns (y, alpha, the t retained singular values)."""
    Y = f.B.T @ f.B
    D, V = np.linalg.eigh((Y + Y.T) / 2.0)
    S = np.sqrt(np.abs(D))
    order = np.argsort(-S, kind="stable")
    St = S[order[:t]]
    Vt_ = V[:, order[:t]]
    Ut = Vt_ / St[None, :]
    coef = Ut.T @ (f.B.T @ rt)
    if alpha is None:
        alpha = upre_alpha(St, coef)
    y = f.Q @ (Vt_ @ (tikhonov_filter(alpha, St) * coef))
    return y, alpha, St


# ---------------------------------------------------------------------------------------
# IRLS


@dataclasses.dataclass
class IRLSParams:
    solver: str = "gkb"          # "gkb" or "rsvd"
    t: int = 10
    tp: int = 11
    beta: float = 0.8            # depth weighting exponent (0.8 gravity, 1.4 magnetic)
    lam: float = 1.0             # focusing norm (1 ~ L1)
    eps2: float = 1e-9
    lower: float = 0.0
    upper: float = 1.0
    kmax: int = 25
    chi2_stop: bool = True       # Eq. (12); False runs exactly kmax iterations
    alphas: Optional[List[float]] = None   # if given, alpha^(k) = alphas[k-1] (no UPRE)


@dataclasses.dataclass
class IRLSReport:
    alphas: List[float]
    chi2: List[float]
    iterations: int


def irls(apply_G: Callable, apply_GT: Callable, d_obs: np.ndarray, sigma: np.ndarray,
         n: int, wz: np.ndarray, p: IRLSParams, omega: Optional[np.ndarray] = None):
    """Sec. 2.3 IRLS loop; apply_G / apply_GT are the unweighted FP64 products."""
    m = d_obs.size
    wd = 1.0 / sigma
    m_prev = np.zeros(n)         # m^(k-1), m^(0) = m_apr = 0
    m_prev2 = np.zeros(n)        # m^(k-2)
    alphas, chi2s = [], []
    for k in range(1, p.kmax + 1):
        wl = np.ones(n) if k == 1 else focusing_weights(m_prev, m_prev2, p.lam, p.eps2)
        winv = 1.0 / (wz * wl)
        rt = wd * (d_obs - apply_G(m_prev))

        def gt(x):
            return wd * apply_G(winv * x)

        def gtt(y):
            return winv * apply_GT(wd * y)

        given = p.alphas[k - 1] if p.alphas is not None else None
        if p.solver == "gkb":
            f = gkb(gt, gtt, rt, p.tp, n)
            U, s, _ = np.linalg.svd(f.B, full_matrices=False)
            alpha = alpha_initial(n, m, s[:p.t]) if k == 1 else None
            z, alpha, _ = gkb_solution(f, p.t, given if given is not None else alpha)
        else:
            f = rsvd(gt, gtt, omega)
            if k == 1:
                _, _, St = rsvd_solution(f, rt, p.t, alpha=1.0)
                alpha = alpha_initial(n, m, St)
            else:
                alpha = None
            z, alpha, _ = rsvd_solution(f, rt, p.t, given if given is not None else alpha)
        m_new = np.clip(m_prev + winv * z, p.lower, p.upper)
        res = wd * (apply_G(m_new) - d_obs)
        chi2 = float(res @ res)
        alphas.append(float(alpha))
        chi2s.append(chi2)
        m_prev2, m_prev = m_prev, m_new
        if p.chi2_stop and chi2 <= m + math.sqrt(2.0 * m):
            break
    return m_prev, IRLSReport(alphas, chi2s, len(alphas))
