"""torch.autograd bridge to the hand-written adjoint of the time step.

``wall_nusselt(phi, H, steps, **cavity)`` returns J = (Nu_f,hot + Nu_s,hot)/2
of the cavity after ``steps`` steps as a differentiable function of the
per-node porosity tensor ``phi`` (shape (ny, nx)) and the scalar tensor
``H``.  The forward call runs the forward pass and the reverse sweep of the
CUDA adjoint together (one C call, ``ltne_adjoint``) and keeps the
gradients; ``backward`` only scales them by the incoming gradient.
"""
from __future__ import annotations

import numpy as np
import torch

from .ltne import Cavity, LTNE_K_ERGUN


class WallNusselt(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, H, steps, segment, storage, cavity_kw):
        ny, nx = phi.shape
        kw = dict(cavity_kw)
        kw.setdefault("permeability", LTNE_K_ERGUN)
        cav = Cavity(nx, ny, storage=storage, porosity_field=1, H=float(H), **kw)
        try:
            J, g, dH = cav.adjoint(phi.detach().double().cpu().numpy().reshape(-1), steps, segment)
        finally:
            cav.close()
        ctx.save_for_backward(g.to(device=phi.device, dtype=phi.dtype),
                              torch.tensor(dH, dtype=H.dtype, device=H.device))
        return torch.tensor(J, dtype=phi.dtype, device=phi.device)

    @staticmethod
    def backward(ctx, gJ):
        g_phi, g_H = ctx.saved_tensors
        return gJ * g_phi, gJ * g_H, None, None, None, None


def wall_nusselt(phi, H, steps, segment=None, storage="f32", **cavity_kw):
    if not torch.is_tensor(H):
        H = torch.tensor(float(H), dtype=torch.float64)
    return WallNusselt.apply(phi, H, int(steps), segment, storage, cavity_kw)
