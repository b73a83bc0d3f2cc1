"""torch.autograd.Function over the library's amplitude-loss gradient kernel.

The loss is L(z, w) = sum_j || |A(w . Q_j z)| - d_j^crop ||^2 with A the PFT of
the PIE context (Section 1: gradient methods need to differentiate through the
PFT). The forward call runs the fused kernel, which recomputes every exit wave
per position instead of storing it and returns L with both gradients
(dL/dRe + i dL/dIm, PyTorch's convention for a real loss of complex inputs);
backward scales them by the incoming gradient.
"""
from __future__ import annotations

import torch


class AmplitudeLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, obj, probe, pie):
        need_probe = bool(probe.requires_grad)
        loss, g_obj, g_probe = pie.amp_loss_grad(obj.detach().contiguous(), probe.detach().contiguous(),
                                                 need_probe_grad=need_probe)
        ctx.save_for_backward(g_obj, g_probe if g_probe is not None else torch.empty(0, device=obj.device))
        ctx.need_probe = need_probe
        return torch.tensor(loss, dtype=torch.float64, device=obj.device)

    @staticmethod
    def backward(ctx, grad_out):
        g_obj, g_probe = ctx.saved_tensors
        scale = grad_out.to(torch.float32)
        gz = g_obj * scale if ctx.needs_input_grad[0] else None
        gw = g_probe * scale if (ctx.needs_input_grad[1] and ctx.need_probe) else None
        return gz, gw, None


def amplitude_loss(obj, probe, pie):
    """L(z, w) through the PFT of `pie` (a PieContext), differentiable in z and w."""
    return AmplitudeLoss.apply(obj, probe, pie)
