"""Differentiable batched solve x = S^-1 b behind torch.autograd.Function.

Forward: setup of every instance's preconditioner blocks and one batched PCG
solve (mixed precision by default).  Backward (hand-written adjoint): with
g = S^-1 (dL/dx), obtained by a second batched PCG solve on the same handle
(S is symmetric, so the same preconditioner serves), the gradients are
    dL/db   = g
    dL/dD_i = -g_i x_i^T
    dL/dO_i = -(g_i x_{i+1}^T + x_i g_{i+1}^T)
since O_i sits at S[i, i+1] and O_i^T at S[i+1, i].  The block outer
products run in the library's adjoint kernel; this module only marshals.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import binding as bb


class _Handle:
    """Owns one batched handle for the lifetime of a forward/backward pair."""

    def __init__(self, Ns, ns, d_off, o_off, D, O, m, alpha, precision, tol_inner):
        self.params, self._keep = bb.make_params(m=m, alpha=alpha, precision=precision, tol_inner=tol_inner)
        st, self.h = bb.bt_setup_batched(Ns, ns, d_off, o_off, D, O, self.params)
        if st != bb.BT_OK:
            if self.h:
                bb.bt_destroy(self.h)
                self.h = None
            raise bb.BTError(st, "bt_setup_batched")
        self.B = len(Ns)

    def solve(self, b, tol, maxit):
        x = torch.zeros_like(b)
        st, it, sts = bb.bt_pcg_solve_batched(self.h, b, x, self.B, tol, maxit)
        if st != bb.BT_OK:
            raise bb.BTError(st, "bt_pcg_solve_batched")
        return x, it

    def close(self):
        if self.h:
            bb.bt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BTSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, O, b, layout, m, alpha, precision, tol, maxit, tol_inner):
        Ns, ns, d_off, o_off = layout
        D = D.contiguous()
        O = O.contiguous()
        b = b.contiguous()
        hd = _Handle(Ns, ns, d_off, o_off, D, O if O.numel() else torch.zeros(1, dtype=D.dtype, device=D.device),
                     m, alpha, precision, tol_inner)
        x, it = hd.solve(b, tol, maxit)
        ctx.hd = hd
        ctx.tol = tol
        ctx.maxit = maxit
        ctx.shapes = (D.shape, O.shape)
        ctx.save_for_backward(x)
        ctx.iters = it
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        hd = ctx.hd
        g, _ = hd.solve(gx.contiguous(), ctx.tol, ctx.maxit)
        gD = torch.empty(ctx.shapes[0], dtype=x.dtype, device=x.device)
        gO = torch.empty(ctx.shapes[1], dtype=x.dtype, device=x.device)
        st = bb.bt_adjoint_blocks(hd.h, x, g, gD, gO if gO.numel() else gD)
        if st != bb.BT_OK:
            raise bb.BTError(st, "bt_adjoint_blocks")
        torch.cuda.current_stream().synchronize()
        hd.close()
        return gD, gO, g, None, None, None, None, None, None, None


def bt_solve(D: torch.Tensor, O: torch.Tensor, b: torch.Tensor, Ns: Sequence[int], ns: Sequence[int],
             d_off: Optional[Sequence[int]] = None, o_off: Optional[Sequence[int]] = None, m: int = 2,
             alpha: Optional[Sequence[float]] = (1.0, 7.0), precision: int = bb.BT_MIXED, tol: float = 1e-8,
             maxit: int = 10000, tol_inner: float = 0.0) -> torch.Tensor:
    """x = S^-1 b for a batch of block-tridiagonal systems packed back to back.

    D: [sum N_k n_k^2], O: [sum (N_k - 1) n_k^2], b: [sum N_k n_k] float64 CUDA
    tensors (row-major blocks, as in include/bt.h).  Differentiable in D, O, b.
    """
    Ns = [int(v) for v in Ns]
    ns = [int(v) for v in ns]
    if d_off is None:
        d_off = np.concatenate([[0], np.cumsum([N * n * n for N, n in zip(Ns, ns)])[:-1]]).tolist()
    if o_off is None:
        o_off = np.concatenate([[0], np.cumsum([max(N - 1, 0) * n * n for N, n in zip(Ns, ns)])[:-1]]).tolist()
    layout = (Ns, ns, [int(v) for v in d_off], [int(v) for v in o_off])
    return BTSolve.apply(D, O, b, layout, m, list(alpha) if alpha is not None else None, precision, tol, maxit,
                         tol_inner)
