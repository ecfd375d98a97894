"""Differentiable products: G X and G^T Y as torch.autograd Functions.

The backward of the forward product is the transpose product and vice versa (App. A:
X^T G^T = (G X)^T), both run by the library's kernels.  For D = diag(r) G diag(c) X:
  dL/dX = diag(c) G^T diag(r) dL/dD,
  dL/dc = sum_b X_b * (G^T diag(r) dL/dD_b),
  dL/dr = sum_b (G diag(c) X_b) * dL/dD_b,
and symmetrically for X = diag(c) G^T diag(r) Y.  This gives, e.g., the weighted misfit
gradient G^T W_d^T W_d (G m - d) of Sec. 2.2 Eq. (5) by back-propagation.
"""
from __future__ import annotations

import torch

__all__ = ["g_matmat", "g_rmatmat"]


class _GMatmat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, colscale, rowscale, op):
        ctx.op = op
        ctx.save_for_backward(X, colscale, rowscale)
        return op.matmat(X.contiguous(), colscale, rowscale)

    @staticmethod
    def backward(ctx, gD):
        op = ctx.op
        X, cs, rs = ctx.saved_tensors
        gD = gD.contiguous()
        gX = gc = gr = None
        need_x, need_c, need_r = ctx.needs_input_grad[:3]
        if need_x or need_c:
            u = op.rmatmat(gD, None, rs)                 # G^T diag(r) gD
            if need_x:
                gX = u * cs if cs is not None else u
            if need_c:
                gc = (X * u).sum(0)
        if need_r:
            gr = (op.matmat(X.contiguous(), cs, None) * gD).sum(0)
        return gX, gc, gr, None


class _GRmatmat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, colscale, rowscale, op):
        ctx.op = op
        ctx.save_for_backward(Y, colscale, rowscale)
        return op.rmatmat(Y.contiguous(), colscale, rowscale)

    @staticmethod
    def backward(ctx, gX):
        op = ctx.op
        Y, cs, rs = ctx.saved_tensors
        gX = gX.contiguous()
        gY = gc = gr = None
        need_y, need_c, need_r = ctx.needs_input_grad[:3]
        if need_y or need_r:
            u = op.matmat(gX, cs, None)                  # G diag(c) gX
            if need_y:
                gY = u * rs if rs is not None else u
            if need_r:
                gr = (Y * u).sum(0)
        if need_c:
            gc = (op.rmatmat(Y.contiguous(), None, rs) * gX).sum(0)
        return gY, gc, gr, None


def _as_block(t):
    return (t.unsqueeze(0), True) if t.dim() == 1 else (t, False)


def g_matmat(op, X, colscale=None, rowscale=None):
    """diag(rowscale) G diag(colscale) X for X of shape (B, n) or (n,), differentiable in
    X, colscale and rowscale."""
    Xb, squeeze = _as_block(X)
    out = _GMatmat.apply(Xb, colscale, rowscale, op)
    return out.squeeze(0) if squeeze else out


def g_rmatmat(op, Y, colscale=None, rowscale=None):
    """diag(colscale) G^T diag(rowscale) Y for Y of shape (B, m) or (m,), differentiable
    in Y, colscale and rowscale."""
    Yb, squeeze = _as_block(Y)
    out = _GRmatmat.apply(Yb, colscale, rowscale, op)
    return out.squeeze(0) if squeeze else out
