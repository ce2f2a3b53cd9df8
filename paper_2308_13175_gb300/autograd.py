"""gp_step as a torch.autograd.Function: the band values are a leaf tensor, the
loss of Eq. 8 is the output, and the hand-written backward of the library is the
gradient.  The forward runs gp_step in loss-only mode; the backward runs gp_step
again (forward recomputed, then the backward), so nothing per query is kept
between the two - at 10^8 queries there is no activation memory to speak of."""
from __future__ import annotations

import torch

from . import binding as gb


class GridPullLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, values, band, rec, B, weights=(1.0, 1.0, 0.005), flags=0):
        loss = torch.zeros(8, dtype=torch.float32, device=values.device)
        gb.gp_step(band, rec, int(B), None, loss, weights, d=values.detach().contiguous(),
                   flags=int(flags) | gb.GP_STEP_LOSS_ONLY)
        ctx.band, ctx.B, ctx.weights, ctx.flags = band, int(B), weights, int(flags)
        ctx.save_for_backward(values, rec)
        return loss[gb.GP_LOSS_TOTAL].clone()

    @staticmethod
    def backward(ctx, grad_out):
        values, rec = ctx.saved_tensors
        grad = torch.empty_like(values)
        loss = torch.zeros(8, dtype=torch.float32, device=values.device)
        gb.gp_step(ctx.band, rec, ctx.B, grad, loss, ctx.weights, d=values.detach().contiguous(), flags=ctx.flags)
        return grad * grad_out, None, None, None, None, None


def gridpull_loss(values, band, rec, B=None, weights=(1.0, 1.0, 0.005), flags=0):
    """L(values) of Eq. 8 over the records, differentiable in ``values``."""
    if B is None:
        B = rec.shape[0]
    return GridPullLoss.apply(values, band, rec, B, weights, flags)
