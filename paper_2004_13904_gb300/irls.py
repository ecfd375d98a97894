"""Binding of the library's IRLS focusing-inversion drivers tf_gkb / tf_rsvd (Sec. 2.2-2.4,
Alg. 1-2, Sec. 3.1), and of its Gram-Schmidt row kernels tf_rows_dot / tf_rows_axpy.

The whole inversion -- every product with G~ = W_d G W^-1 (Sec. 2.5 Eq. (10)), the
re-orthogonalisation, the projected solves, UPRE and the IRLS weights -- runs below the
C ABI (csrc/tf_irls.cu); this module only marshals arguments and results.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional

import torch

from . import _lib

__all__ = ["IRLSOptions", "IRLSResult", "invert_native", "rows_dot", "rows_axpy"]


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dt_code(t: torch.Tensor) -> int:
    return _lib.TF_F32 if t.dtype == torch.float32 else _lib.TF_F64


def rows_dot(A: torch.Tensor, k: int, x: torch.Tensor) -> torch.Tensor:
    """tf_rows_dot: y[j] = A_j . x for the first k rows of A (FP64 result)."""
    y = torch.empty(max(k, 1), dtype=torch.float64, device=x.device)
    _lib.check(_lib.lib().tf_rows_dot(_dt_code(A), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                      k, x.numel(), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(y.data_ptr()), _stream()))
    return y[:k]


def rows_axpy(A: torch.Tensor, k: int, c: torch.Tensor, x: torch.Tensor) -> None:
    """tf_rows_axpy: x -= sum_j c[j] A_j over the first k rows of A (c is FP64)."""
    _lib.check(_lib.lib().tf_rows_axpy(_dt_code(A), ctypes.c_void_p(A.data_ptr()), A.stride(0),
                                       k, x.numel(), ctypes.c_void_p(c.data_ptr()),
                                       ctypes.c_void_p(x.data_ptr()), _stream()))


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
