"""torch.autograd.Function over the library's solve, logdet and adjoint.

The loss terms sum_k w_k^T x_k and log det A, with x = A^{-1} b and A given by
its stored lower entries, get their gradients from the library's adjoint
(chol_adjoint): dl/db = A^{-1} (dl/dx) and dl/da_ij from -xbar x^T plus the
selected inverse. The Python side only passes pointers and streams.
"""
from __future__ import annotations

import torch

from . import CholError, SparseCholesky, chol_adjoint


class SolveLogdet(torch.autograd.Function):
    """(values, b) -> (x = A^{-1} b, log det A), differentiable in both inputs.

    ``solver`` is a SparseCholesky analysed on A's pattern (binary64 mode);
    ``values`` is float64 on the GPU in the analysed entry order; ``b`` is
    n x nrhs (any layout) or n.
    """

    @staticmethod
    def forward(ctx, values, b, solver: SparseCholesky):
        solver.factor(values)
        x = solver.solve(b if b.dim() == 2 else b.unsqueeze(1))
        ld = torch.tensor(solver.logdet(), dtype=torch.float64, device=values.device)
        ctx.solver = solver
        ctx.b_dim = b.dim()
        ctx.save_for_backward(x)
        return (x if b.dim() == 2 else x.squeeze(1)), ld

    @staticmethod
    def backward(ctx, gx, gld):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        n, nrhs = x.shape
        w = torch.zeros_like(x) if gx is None else (gx if gx.dim() == 2 else gx.unsqueeze(1))
        w = w.t().contiguous().t()                       # column-major n x nrhs
        xc = x.t().contiguous().t()
        alpha = 0.0 if gld is None else float(gld)
        bbar = torch.empty_like(xc)
        grad = torch.empty(solver.info.nnz_a, dtype=torch.float64, device=x.device)
        rc = chol_adjoint(solver.h, w, xc, nrhs, alpha, bbar, grad, torch.cuda.current_stream())
        if rc:
            raise CholError(rc, "chol_adjoint")
        gb = bbar if ctx.b_dim == 2 else bbar.squeeze(1)
        return grad, gb, None


def solve_logdet(values, b, solver):
    return SolveLogdet.apply(values, b, solver)
