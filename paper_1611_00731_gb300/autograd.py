"""torch.autograd binding of the assembly map V -> H (Sec. 4 eq. disceig3d).

H depends on the local potential at the quadrature points only through the
term sum_q w_q V_q b_q b_q^T of every element, so H(V) is affine in V and
its vector-Jacobian product for a cotangent Hbar on the CSR pattern is
    dL/dV_q = w_q b_q^T Hbar_e b_q,   L = sum_ij Hbar_ij H_ij,
which is what pufe_assemble_HV_adjoint computes (the hand-written backward
kernel).  With Hbar_ij = sum_n f_n c_in c_jn for fixed states c_n this is the
Hellmann-Feynman derivative of the band energy sum_n f_n c_n^T H c_n, i.e.
w_q times the density of the states at the point (Sec. 3 eq. rhoe).

Both directions run in the library's kernels; this module only moves tensors.
"""
from __future__ import annotations

import torch

from . import pufe


class AssembleH(torch.autograd.Function):
    """H values (nnz, float64, on the context's CSR pattern) from V (n_q)."""

    @staticmethod
    def forward(fctx, V, ctx, prec):
        H = torch.empty(ctx.nnz, dtype=torch.float64, device=V.device)
        ctx.pufe_assemble_HS(V.detach().contiguous(), H, None, prec=prec)
        fctx.pctx = ctx
        fctx.prec = prec
        return H

    @staticmethod
    def backward(fctx, grad_H):
        ctx = fctx.pctx
        Vbar = torch.empty(ctx.n_q, dtype=torch.float64, device=grad_H.device)
        ctx.pufe_assemble_HV_adjoint(grad_H.contiguous(), Vbar, prec=fctx.prec)
        return Vbar, None, None


def assemble_H(ctx, V, prec=pufe.PUFE_FP64):
    """Differentiable H(V): the context must be tabulated in `prec`."""
    return AssembleH.apply(V, ctx, prec)
