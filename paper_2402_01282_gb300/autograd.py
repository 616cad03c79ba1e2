"""torch.autograd bindings of the wavelet transforms (Sec. 4.3: the transforms are
differentiable).  The backward pass of each transform is the library's hand-written adjoint
(s2w_forward_adjoint / s2w_inverse_adjoint): the transposed DFTs, contraction, products and
quadrature, with the Wigner-d values recomputed by the recursion instead of stored.  For a
linear map y = A x PyTorch hands backward the gradient g = dLoss/dy (conjugate-Wirtinger
convention for complex tensors) and wants A^H g, which is what the adjoints compute.

    plan = Plan(L, N, lam, J0, reality=True, batch=B)
    wav, scal = analysis(f, plan)        # f: [B, L, 2L-1] float64 on the GPU, requires_grad
    f2 = synthesis(wav, scal, plan)
"""
from __future__ import annotations

import torch


class _Analysis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, plan):
        f = f.contiguous()
        wav, scal = plan.empty_wav(), plan.empty_scal()
        plan.forward(f, wav, scal)
        ctx.plan = plan
        return wav, scal

    @staticmethod
    def backward(ctx, gwav, gscal):
        plan = ctx.plan
        if gwav is None:
            gwav = torch.zeros_like(plan.empty_wav())
        if gscal is None:
            gscal = torch.zeros_like(plan.empty_scal())
        gf = plan.empty_map()
        plan.forward_adjoint(gwav.contiguous(), gscal.contiguous(), gf)
        return gf, None


class _Synthesis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, wav, scal, plan):
        f = plan.empty_map()
        plan.inverse(wav.contiguous(), scal.contiguous(), f)
        ctx.plan = plan
        return f

    @staticmethod
    def backward(ctx, gf):
        plan = ctx.plan
        gwav, gscal = plan.empty_wav(), plan.empty_scal()
        plan.inverse_adjoint(gf.contiguous(), gwav, gscal)
        return gwav, gscal, None


def analysis(f: torch.Tensor, plan):
    """Differentiable s2w_forward: f [batch, L, 2L-1] -> (wav [batch, wav_elems], scal)."""
    return _Analysis.apply(f, plan)


def synthesis(wav: torch.Tensor, scal: torch.Tensor, plan):
    """Differentiable s2w_inverse: (wav, scal) -> f [batch, L, 2L-1]."""
    return _Synthesis.apply(wav, scal, plan)
