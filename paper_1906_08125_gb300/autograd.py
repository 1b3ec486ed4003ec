"""torch.autograd bridge of pic_adjoint.

``collected_charge(pic, E0, wf, n_steps)`` returns the charge collected
through Gamma_1 over ``n_steps`` PIC steps of the context ``pic`` as a tensor
that is differentiable in the applied field(s) ``E0`` (one per replica) and
the per-face work functions ``wf``.  The forward call runs the steps (the
context advances by ``n_steps``) and obtains the gradient in the same
pic_adjoint call (forward run with checkpoints every ``ckpt_every`` steps,
then the reverse pass); backward only scales it.  The derivative is that of
the frozen-decision smooth model documented at pic_adjoint in picfem.h.
"""
from __future__ import annotations

import numpy as np
import torch


class CollectedCharge(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E0, wf, pic, n_steps, ckpt_every):
        pic.set_applied_field(E0.detach().double().cpu().numpy())
        pic.set_work_function(np.ascontiguousarray(wf.detach().double().cpu().numpy()))
        Q, gE0, gwf = pic.adjoint(int(n_steps), int(ckpt_every))
        ctx.save_for_backward(
            torch.as_tensor(gE0, dtype=E0.dtype, device=E0.device).reshape(E0.shape),
            torch.as_tensor(gwf, dtype=wf.dtype, device=wf.device).reshape(wf.shape))
        return torch.tensor(Q, dtype=torch.float64, device=E0.device)

    @staticmethod
    def backward(ctx, gQ):
        gE0, gwf = ctx.saved_tensors
        return (gQ.to(gE0.dtype) * gE0, gQ.to(gwf.dtype) * gwf, None, None, None)


def collected_charge(pic, E0, wf, n_steps, ckpt_every=20):
    """Differentiable collected charge [C] over n_steps steps of ``pic``."""
    return CollectedCharge.apply(E0, wf, pic, n_steps, ckpt_every)
