"""Compliance c(E) = u^T A(E) u as a torch.autograd.Function.

For a fixed nodal field u the compliance is linear in the per-cell
coefficients (Eq. assembly: A = sum_K coef_K A^K / coef_K), so its gradient is
the vector of cell energies per unit coefficient, dc/dcoef_K = u_K^T (A^K /
coef_K) u_K. Both the forward value and the backward gradient come from the
adjoint kernel of libfeasm (fe_assemble_adjoint); u is treated as a constant
(no gradient with respect to u).
"""
from __future__ import annotations

import torch

from . import feasm


class Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coef: torch.Tensor, u: torch.Tensor, space: "feasm.FESpace", prec: str = "fp64"):
        c = torch.empty(1, dtype=torch.float64, device=coef.device)
        g = torch.empty(space.n_cells, dtype=torch.float64, device=coef.device)
        feasm.fe_assemble_adjoint(space.handle, u, coef, 1.0, g, c, feasm.PRECISIONS[prec])
        ctx.space = space
        ctx.prec = prec
        ctx.save_for_backward(coef, u)
        return c[0]

    @staticmethod
    def backward(ctx, grad_c: torch.Tensor):
        coef, u = ctx.saved_tensors
        g = torch.empty(ctx.space.n_cells, dtype=torch.float64, device=coef.device)
        feasm.fe_assemble_adjoint(ctx.space.handle, u, None, float(grad_c), g, None, feasm.PRECISIONS[ctx.prec])
        return g, None, None, None


def compliance(coef: torch.Tensor, u: torch.Tensor, space: "feasm.FESpace", prec: str = "fp64") -> torch.Tensor:
    return Compliance.apply(coef, u, space, prec)
