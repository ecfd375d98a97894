"""IRLS focusing inversion on the GPU with the GKB and RSVD solvers (Sec. 2.2-2.4,
Alg. 1-2, Sec. 3.1).

Every product with G~ = W_d G W^-1 (Sec. 2.5 Eq. (10)) is one library call with
colscale = W^-1 and rowscale = W_d, so the diagonal scalings cost nothing extra.  Block
products serve the RSVD (Alg. 2: t_p columns at a time).  Re-orthogonalisation against
the stored bases runs in the library's FP64-accumulating row kernels (tf_rows_dot /
tf_rows_axpy): either modified Gram-Schmidt in the order of Alg. 1, or two classical
passes (CGS2), which matches it to rounding and moves each basis once per pass.  QR
factors of the tall RSVD blocks come from cuSOLVER (through torch.linalg.qr); the small
projected SVD / eigen-decomposition, UPRE and the Tikhonov filter run in FP64 on the
host.

Reading of the paper's silent points (the same reading as the CPU reference): UPRE for
whitened noise on the t retained terms, minimised over 200 log-spaced points on
[max(s_t, 1e-14 s_1)/10, s_1] then refined by golden-section search between the grid
neighbours of the best point; alpha^(1) from Eq. (11) with the mean over the t retained
singular values above 1e-14 s_1; W_L^(1) = I and W_L^(k) from the two previous iterates.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time
from typing import List, Optional

import numpy as np
import torch

from . import _lib

__all__ = ["IRLSOptions", "IRLSResult", "invert", "invert_native", "gkb_factor", "rsvd_factor",
           "upre_value", "choose_alpha"]

_GOLD = (math.sqrt(5.0) - 1.0) / 2.0


# ------------------------------------------------------------------------ regularisation

def upre_value(alpha, s: np.ndarray, coef: np.ndarray):
    """UPRE(alpha) on the retained terms, whitened noise, alpha-independent terms dropped.
    alpha may be a scalar or an array."""
    a = np.asarray(alpha, np.float64)[..., None]
    s2 = s * s
    phi = s2 / (s2 + a * a)
    val = ((1.0 - phi) ** 2 * coef * coef).sum(-1) + 2.0 * phi.sum(-1) - s.size
    return val if val.ndim else float(val)


def choose_alpha(s: np.ndarray, coef: np.ndarray) -> float:
    """argmin UPRE: 200-point log grid, then golden-section search in log alpha."""
    s = np.asarray(s, np.float64)
    coef = np.asarray(coef, np.float64)
    lo = math.log(max(s[-1], 1e-14 * s[0]) / 10.0)
    hi = math.log(s[0])
    grid = np.exp(np.linspace(lo, hi, 200))
    vals = upre_value(grid, s, coef)
    k = int(np.argmin(vals))
    left, right = math.log(grid[max(k - 1, 0)]), math.log(grid[min(k + 1, 199)])
    x1 = right - _GOLD * (right - left)
    x2 = left + _GOLD * (right - left)
    f1, f2 = upre_value(math.exp(x1), s, coef), upre_value(math.exp(x2), s, coef)
    for _ in range(80):
        if f1 <= f2:
            right, x2, f2 = x2, x1, f1
            x1 = right - _GOLD * (right - left)
            f1 = upre_value(math.exp(x1), s, coef)
        else:
            left, x1, f1 = x1, x2, f2
            x2 = left + _GOLD * (right - left)
            f2 = upre_value(math.exp(x2), s, coef)
    mid = math.exp(0.5 * (left + right))
    return mid if upre_value(mid, s, coef) <= vals[k] else float(grid[k])


def _alpha_start(n: int, m: int, s: np.ndarray) -> float:
    keep = s[s > 1e-14 * s[0]]
    return (n / m) ** 3.5 * float(s[0]) / float(keep.mean())


# ------------------------------------------------------------------------ GPU helpers

def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dt_code(t: torch.Tensor) -> int:
    return _lib.TF_F32 if t.dtype == torch.float32 else _lib.TF_F64


def _rows_dot(A: torch.Tensor, k: int, x: torch.Tensor) -> torch.Tensor:
    y = torch.empty(max(k, 1), dtype=torch.float64, device=x.device)
    _lib.check(_lib.lib().tf_rows_dot(_dt_code(A), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                      k, x.numel(), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), _stream()))
    return y[:k]


def _rows_axpy(A: torch.Tensor, k: int, c: torch.Tensor, x: torch.Tensor) -> None:
    _lib.check(_lib.lib().tf_rows_axpy(_dt_code(A), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                       k, x.numel(), ctypes.c_void_p(c.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), _stream()))


def _orthogonalise(V: torch.Tensor, k: int, x: torch.Tensor, method: str) -> None:
    """x <- x minus its components along the first k rows of V (orthonormal)."""
    if k == 0:
        return
    if method == "mgs":
        for j in range(k):
            row = V[j:j + 1]
            _rows_axpy(row, 1, _rows_dot(row, 1, x), x)
    else:
        for _ in range(2):
            _rows_axpy(V, k, _rows_dot(V, k, x), x)


def _combine(V: torch.Tensor, w: np.ndarray, length: int) -> torch.Tensor:
    """sum_j w[j] V_j (FP64 accumulation) in V's dtype."""
    out = torch.zeros(length, dtype=V.dtype, device=V.device)
    c = torch.tensor(-np.asarray(w, np.float64), device=V.device)
    _rows_axpy(V, len(w), c, out)
    return out


def _norm64(x: torch.Tensor) -> float:
    return float(torch.linalg.vector_norm(x, dtype=torch.float64))


# ------------------------------------------------------------------------ solvers

@dataclasses.dataclass
class GKB:
    A: torch.Tensor       # t_p x n, row j = column j of A
    B: np.ndarray         # (t_p+1) x t_p, FP64
    rnorm: float


def gkb_factor(op, rt: torch.Tensor, winv: torch.Tensor, wd: torch.Tensor, tp: int,
               reorth: str = "cgs2") -> GKB:
    """Alg. 1: G~ A = H B, G~ = diag(wd) G diag(winv), with re-orthogonalisation.  The
    norms stay on the device, so the loop does not wait for the host."""
    n, m, dt, dev = op.n, op.m, op.dtype, op.device
    A = torch.zeros((tp, n), dtype=dt, device=dev)
    H = torch.zeros((tp + 1, m), dtype=dt, device=dev)
    diag = torch.zeros(tp, dtype=torch.float64, device=dev)      # B(i, i) = gamma_i
    sub = torch.zeros(tp, dtype=torch.float64, device=dev)       # B(i+1, i) = beta_{i+1}
    beta = torch.linalg.vector_norm(rt, dtype=torch.float64)
    rnorm = float(beta)
    H[0] = rt / beta.to(dt)
    a = torch.zeros(n, dtype=dt, device=dev)
    for i in range(tp):
        b = op.rmatvec(H[i], colscale=winv, rowscale=wd)
        b -= beta.to(dt) * a
        _orthogonalise(A, i, b, reorth)
        gamma = torch.linalg.vector_norm(b, dtype=torch.float64)
        a = b / gamma.to(dt)
        A[i] = a
        diag[i] = gamma
        c = op.matvec(a, colscale=winv, rowscale=wd)
        c -= gamma.to(dt) * H[i]
        _orthogonalise(H, i + 1, c, reorth)
        beta = torch.linalg.vector_norm(c, dtype=torch.float64)
        H[i + 1] = c / beta.to(dt)
        sub[i] = beta
    B = np.zeros((tp + 1, tp))
    idx = np.arange(tp)
    B[idx, idx] = diag.cpu().numpy()
    B[idx + 1, idx] = sub.cpu().numpy()
    return GKB(A, B, rnorm)


# Projected problems up to this size use a dense LAPACK SVD on the host; larger GKB
# bidiagonals use the tridiagonal route below, larger RSVD Gram matrices cuSOLVER.
_HOST_MAX = 512


def _lower_to_upper(gam: np.ndarray, bet: np.ndarray):
    """Givens rotations Q^T B = [R; 0] turning the lower bidiagonal (t_p+1) x t_p matrix
    (diagonal gam, subdiagonal bet) into an upper bidiagonal R (diagonal d, superdiagonal
    e); also returns q = Q^T e_1, whose first t_p entries are the first row of Q's leading
    columns."""
    n = gam.size
    d = np.empty(n)
    e = np.empty(max(n - 1, 0))
    q = np.zeros(n + 1)
    q[0] = 1.0
    a = gam[0]
    for i in range(n):
        r = math.hypot(a, bet[i])
        c, s_ = a / r, bet[i] / r
        d[i] = r
        if i + 1 < n:
            e[i] = s_ * gam[i + 1]
            a = c * gam[i + 1]
        qi, qj = q[i], q[i + 1]
        q[i], q[i + 1] = c * qi + s_ * qj, c * qj - s_ * qi
    return d, e, q


def bidiag_svd(B: np.ndarray):
    """SVD pieces of the GKB bidiagonal B needed by the solve: (first row of U, singular
    values descending, V^T).  Small B: dense LAPACK.  Large B: Givens reduction to an
    upper bidiagonal R, then the eigen-decomposition of the 2n x 2n Golub-Kahan
    tridiagonal matrix (zero diagonal, off-diagonals d1, e1, d2, ...; LAPACK dstevd),
    whose eigenvectors for +sigma interleave (v_1, u_1, v_2, u_2, ...)/sqrt(2)."""
    tp = B.shape[1]
    if tp <= _HOST_MAX:
        U, s, Vh = np.linalg.svd(B, full_matrices=False)
        return U[0], s, Vh
    from scipy.linalg import lapack
    gam = np.diagonal(B).copy()
    bet = np.diagonal(B, -1).copy()
    d, e, q = _lower_to_upper(gam, bet)
    off = np.empty(2 * tp - 1)
    off[0::2] = d
    off[1::2] = e
    w, Z, info = lapack.dstevd(np.zeros(2 * tp), off, compute_v=1)
    if info != 0:
        raise RuntimeError(f"dstevd failed ({info})")
    top = np.argsort(-w, kind="stable")[:tp]
    Z = Z[:, top] * math.sqrt(2.0)
    V, Ur = Z[0::2, :], Z[1::2, :]
    return q[:tp] @ Ur, w[top], V.T


def gkb_solve(f: GKB, t: int, n: int, alpha: Optional[float] = None, svd=None):
    u1, s, Vh = svd if svd is not None else bidiag_svd(f.B)
    coef = f.rnorm * u1
    if alpha is None:
        alpha = choose_alpha(s[:t], coef[:t])
    w = Vh.T @ (coef * s / (s * s + alpha * alpha))
    return _combine(f.A, w, n), alpha, s


@dataclasses.dataclass
class RSVD:
    Q: torch.Tensor       # t_p x n, rows = columns of the last QR factor
    Bt: torch.Tensor      # t_p x m, rows = columns of B = G~ Q


def _orthonormal_rows(Y: torch.Tensor) -> torch.Tensor:
    """Rows of the result are an orthonormal basis of the rows of Y (economic QR)."""
    return torch.linalg.qr(Y.T, mode="reduced").Q.T.contiguous()


def rsvd_factor(op, omega: torch.Tensor, winv: torch.Tensor, wd: torch.Tensor) -> RSVD:
    """Alg. 2 with one power iteration; omega (t_p x m) is the Gaussian test matrix."""
    kw = dict(colscale=winv, rowscale=wd)
    Q = _orthonormal_rows(op.rmatmat(omega, **kw))     # Y = Omega G~,  [Q,~] = qr(Y^T)
    Q1 = _orthonormal_rows(op.matmat(Q, **kw))         # Y = G~ Q,      [Q,~] = qr(Y)
    Q2 = _orthonormal_rows(op.rmatmat(Q1, **kw))       # Y = Q^T G~,    [Q,~] = qr(Y^T)
    return RSVD(Q2, op.matmat(Q2, **kw))               # B = G~ Q


def rsvd_solve(f: RSVD, rt: torch.Tensor, t: int, n: int, alpha: Optional[float] = None):
    Bt = f.Bt.double()
    M = Bt @ Bt.T
    if M.shape[0] <= _HOST_MAX:
        M = M.cpu().numpy()
        D, V = np.linalg.eigh((M + M.T) / 2.0)
    else:
        D, V = torch.linalg.eigh((M + M.T) / 2.0)
        D, V = D.cpu().numpy(), V.cpu().numpy()
    S = np.sqrt(np.abs(D))
    idx = np.argsort(-S, kind="stable")[:t]
    St, Vt = S[idx], V[:, idx]
    btr = (Bt @ rt.double()).cpu().numpy()
    coef = (Vt / St[None, :]).T @ btr
    if alpha is None:
        alpha = choose_alpha(St, coef)
    w = Vt @ (coef * St / (St * St + alpha * alpha))
    return _combine(f.Q, w, n), alpha, St


# ------------------------------------------------------------------------ IRLS

@dataclasses.dataclass
class IRLSOptions:
    solver: str = "gkb"           # "gkb" (Alg. 1) or "rsvd" (Alg. 2)
    t: int = 10                   # retained terms
    tp: int = 11                  # projected size
    beta: float = 0.8             # depth weighting exponent
    lam: float = 1.0              # focusing norm
    eps2: float = 1e-9
    lower: float = 0.0
    upper: float = 1.0
    kmax: int = 25
    chi2_stop: bool = True        # stop when chi^2 <= m + sqrt(2m) (Eq. (12))
    reorth: str = "cgs2"          # "cgs2" or "mgs" (GKB only)
    alphas: Optional[List[float]] = None   # fixed alpha^(k) = alphas[k-1] (skips UPRE)


@dataclasses.dataclass
class IRLSResult:
    model: torch.Tensor
    alphas: List[float]
    chi2: List[float]
    seconds: List[float]
    factor_seconds: List[float] = dataclasses.field(default_factory=list)


def depth_weight_vector(grid, beta: float, dtype, device) -> torch.Tensor:
    """W_z diagonal: (mean layer depth below the stations)^(-beta) per layer."""
    z = np.asarray(grid.z_edges, np.float64) - grid.station_z
    per_layer = (0.5 * (z[1:] + z[:-1])) ** (-beta)
    w = np.repeat(per_layer, grid.nx * grid.ny)
    return torch.tensor(w, dtype=dtype, device=device)


def invert(op, grid, d_obs: torch.Tensor, sigma: torch.Tensor, opts: IRLSOptions,
           omega: Optional[torch.Tensor] = None) -> IRLSResult:
    """Focusing inversion m* of Eq. (4) by IRLS with the chosen projected solver."""
    n, m = op.n, op.m
    dt, dev = op.dtype, op.device
    wd = (1.0 / sigma).to(dt)
    wz = depth_weight_vector(grid, opts.beta, dt, dev)
    m1 = torch.zeros(n, dtype=dt, device=dev)          # m^(k-1)
    m2 = torch.zeros(n, dtype=dt, device=dev)          # m^(k-2)
    res = IRLSResult(m1, [], [], [], [])
    for k in range(1, opts.kmax + 1):
        t0 = time.perf_counter()
        if k == 1:
            wl = torch.ones(n, dtype=dt, device=dev)
        else:
            wl = ((m1 - m2) ** 2 + opts.eps2) ** ((opts.lam - 2.0) / 4.0)
        winv = 1.0 / (wz * wl)
        rt = wd * (d_obs - op.matvec(m1))
        fixed = opts.alphas[k - 1] if opts.alphas is not None else None
        if opts.solver == "gkb":
            f = gkb_factor(op, rt, winv, wd, opts.tp, opts.reorth)
            torch.cuda.synchronize()
            res.factor_seconds.append(time.perf_counter() - t0)
            svd = bidiag_svd(f.B)
            a0 = fixed
            if k == 1 and a0 is None:
                a0 = _alpha_start(n, m, svd[1][:opts.t])
            z, alpha, _ = gkb_solve(f, opts.t, n, a0, svd)
        else:
            f = rsvd_factor(op, omega, winv, wd)
            torch.cuda.synchronize()
            res.factor_seconds.append(time.perf_counter() - t0)
            a0 = fixed
            if k == 1 and a0 is None:
                _, _, St = rsvd_solve(f, rt, opts.t, n, alpha=1.0)
                a0 = _alpha_start(n, m, St)
            z, alpha, _ = rsvd_solve(f, rt, opts.t, n, a0)
        m_new = torch.clamp(m1 + winv * z, opts.lower, opts.upper)
        r = wd * (op.matvec(m_new) - d_obs)
        chi2 = _norm64(r) ** 2
        torch.cuda.synchronize()
        res.alphas.append(float(alpha))
        res.chi2.append(chi2)
        res.seconds.append(time.perf_counter() - t0)
        m2, m1 = m1, m_new
        if opts.chi2_stop and chi2 <= m + math.sqrt(2.0 * m):
            break
    res.model = m1
    return res


def invert_native(op, d_obs: torch.Tensor, sigma: torch.Tensor, opts: IRLSOptions,
                  omega: Optional[torch.Tensor] = None) -> IRLSResult:
    """The same inversion through the library's C drivers tf_gkb / tf_rsvd (the whole
    IRLS loop runs below the C ABI; the depth weights come from the operator's grid)."""
    n, m = op.n, op.m
    d_obs = d_obs.to(op.dtype).contiguous()
    sigma = sigma.to(op.dtype).contiguous()
    out = torch.empty(n, dtype=op.dtype, device=op.device)
    fixed = None
    if opts.alphas is not None:
        if len(opts.alphas) < opts.kmax:
            raise ValueError(f"alphas has {len(opts.alphas)} entries, kmax is {opts.kmax}")
        fixed = (ctypes.c_double * opts.kmax)(*[float(a) for a in opts.alphas[:opts.kmax]])
    p = _lib.tf_irls_params(opts.t, opts.tp, opts.beta, opts.lam, opts.eps2, opts.lower,
                            opts.upper, opts.kmax, 1 if opts.chi2_stop else 0,
                            1 if opts.reorth == "mgs" else 0,
                            ctypes.cast(fixed, ctypes.POINTER(ctypes.c_double)) if fixed else None)
    alphas = (ctypes.c_double * opts.kmax)()
    chi2 = (ctypes.c_double * opts.kmax)()
    secs = (ctypes.c_double * opts.kmax)()
    rep = _lib.tf_irls_report(0, alphas, chi2, secs)
    L = _lib.lib()
    dp = ctypes.c_void_p
    if opts.solver == "gkb":
        st = L.tf_gkb(op._h, ctypes.byref(p), dp(d_obs.data_ptr()), dp(sigma.data_ptr()),
                      dp(out.data_ptr()), ctypes.byref(rep), _stream())
    else:
        if omega is None:
            raise ValueError("the RSVD solver needs omega (t_p x m)")
        om = omega.to(op.dtype).contiguous()
        st = L.tf_rsvd(op._h, ctypes.byref(p), dp(d_obs.data_ptr()), dp(sigma.data_ptr()),
                       dp(om.data_ptr()), dp(out.data_ptr()), ctypes.byref(rep), _stream())
    _lib.check(st)
    k = rep.iterations
    return IRLSResult(out, list(alphas[:k]), list(chi2[:k]), list(secs[:k]))
