"""torch.autograd.Function over tersoff_param_grad: the fitness loss of every parameter set as a
differentiable function of the parameters (the gradient polish of the GA's best individuals)."""
from __future__ import annotations

import torch

from . import binding


class TersoffLoss(torch.autograd.Function):
    """L[p] = loss of parameter set p over the context's configurations and targets.

    forward(params [P][6] float64 CUDA, ctx, targets, w, loss) -> L [P]; backward gives
    dL/dparams = grad_L[p] * dL[p]/dx from the library's adjoint kernel.
    """

    @staticmethod
    def forward(fctx, params, ctx: binding.Context, targets: dict, w=(1.0, 1.0, 1.0), loss: int = binding.LOSS_SQ):
        L, dL = ctx.param_grad(params.detach().contiguous(), targets, w=w, loss=loss)
        fctx.save_for_backward(dL)
        return L

    @staticmethod
    def backward(fctx, grad_L):
        (dL,) = fctx.saved_tensors
        return grad_L[:, None] * dL, None, None, None, None
