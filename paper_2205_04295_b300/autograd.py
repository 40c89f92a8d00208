"""torch.autograd.Function around the library's differentiable forward model.

forward  -> pty_loss       (the loss only; nothing of the far field is kept)
backward -> pty_loss_grad  (recomputes each patch's far field and runs the
                            hand-written adjoint)
Gradients follow PyTorch's convention for complex tensors (dL/dRe + i dL/dIm),
so optimisers can step O, P and the positions directly.
"""
import torch

from . import pty


class AmplitudeLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, O, P, pos, problem, delta):
        O, P, pos = O.contiguous(), P.contiguous(), pos.contiguous()
        loss = problem.loss(O, P, pos, delta)
        ctx.save_for_backward(O, P, pos)
        ctx.problem, ctx.delta = problem, delta
        return loss[0]

    @staticmethod
    def backward(ctx, grad_out):
        O, P, pos = ctx.saved_tensors
        _, gO, gP, gpos = ctx.problem.loss_grad(O, P, pos, ctx.delta)
        return grad_out * gO, grad_out * gP, grad_out * gpos, None, None


def amplitude_loss(problem, O, P, pos, delta=1.0):
    """L = sum_j sum_u (sqrt(sum_p |F(P_p o_j)|^2 + delta) - sqrt(I_j))^2,
    differentiable with respect to O, P and pos (CUDA tensors)."""
    return AmplitudeLoss.apply(O, P, pos, problem, delta)
