"""Differentiable PackSELL products and solves (torch.autograd Functions).

Argument marshalling around the C ABI: every product, transpose, pattern
gradient and solve runs in the CUDA library.

* :func:`spmv` - y = A x. Backward (packsell_spmv_backward): dx = A^T dy and,
  when the CSR values A was encoded from require grad, dL/da_ij = dy_i x_j on
  the pattern; the quantiser is passed straight through (dq(v)/dv = 1).
* :func:`solve` - x = A^-1 b for SPD A given as CSR (rowptr, col, values) on
  the device, by packsell_pcg (FP64 PCG, or the mixed-precision inner-outer
  CG with a PackSELL inner matrix). Backward (packsell_pcg_backward): one
  adjoint solve A lam = dL/dx (A is symmetric), then dL/db = lam and
  dL/da_ij = -lam_i x_j on the pattern. Gradients with respect to parameters that
  build the values (face coefficients, say) follow by autograd through the
  user's own assembly of the values.
"""
from __future__ import annotations

import torch

from . import packsell as ps


class _SpMV(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, x, A):
        ctx.A = A
        ctx.val_dtype = val.dtype
        ctx.save_for_backward(x)
        return ps.packsell_spmv(A, x)

    @staticmethod
    def backward(ctx, dy):
        (x,) = ctx.saved_tensors
        need_dval, need_dx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_dval or need_dx):
            return None, None, None
        dx, dval = ps.packsell_spmv_backward(ctx.A, x, dy.contiguous().float(),
                                             need_dx=need_dx, need_dval=need_dval)
        if dval is not None:
            dval = dval.to(ctx.val_dtype)
        return dval, dx, None


def spmv(A: ps.PackSELLMatrix, x: torch.Tensor, val: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable y = A x. ``val``: the CSR values A was encoded from (its
    gradient needs A encoded with keep_rowptr=True); omit it to differentiate
    with respect to x only."""
    if val is None:
        val = torch.empty(0, device=x.device)
    return _SpMV.apply(val, x, A)


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, val, b, rowptr, col, opts):
        n = rowptr.numel() - 1
        A64 = ps.packsell_encode(rowptr, col, val.detach().double().contiguous(), n, n,
                                 fmt="sell_f64", keep_rowptr=True)
        Ain = None
        if opts["m_in"] > 0:
            Ain = ps.packsell_encode(rowptr, col, val.detach().contiguous(), n, n,
                                     fmt=opts["fmt"], D=opts["D"])
        M = ps.packsell_inv_diag(A64) if opts["jacobi"] else None
        kw = dict(A_inner=Ain, inv_diag=M, m_in=opts["m_in"], rtol=opts["rtol"],
                  max_iters=opts["max_iters"])
        x, info = ps.packsell_pcg(A64, b.detach().double().contiguous(), **kw)
        ctx.A64, ctx.kw = A64, kw
        ctx.val_dtype, ctx.b_dtype = val.dtype, b.dtype
        ctx.info = info
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, g):
        (x,) = ctx.saved_tensors
        need_dA = ctx.needs_input_grad[0]
        lam, dA, _ = ps.packsell_pcg_backward(ctx.A64, x, g.detach().double().contiguous(),
                                              need_dA=need_dA, **ctx.kw)
        dval = dA.to(ctx.val_dtype) if need_dA else None
        db = lam.to(ctx.b_dtype) if ctx.needs_input_grad[1] else None
        return dval, db, None, None, None


def solve(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, b: torch.Tensor, *,
          m_in: int = 0, fmt: str = "fp16", D: int = 15, jacobi: bool = True,
          rtol: float = 1e-12, max_iters: int = 5000) -> torch.Tensor:
    """Differentiable x = A^-1 b (A SPD, CSR on the device, float64 result)."""
    opts = {"m_in": int(m_in), "fmt": fmt, "D": int(D), "jacobi": bool(jacobi),
            "rtol": float(rtol), "max_iters": int(max_iters)}
    return _Solve.apply(val, b, rowptr, col, opts)
