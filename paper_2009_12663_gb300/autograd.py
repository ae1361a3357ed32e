"""The misfit of Eq. A1 as a differentiable torch function.

forward(): the forward simulations and the misfit only (gbfwi_misfit).
backward(): the adjoint simulations (gbfwi_adjoint_gradient), which replay
the forward field from snapshots every `ckpt_every` steps instead of keeping
every wavefield level, correlate it with the adjoint field (the discrete
form of Eqs. A16-A18) and return d misfit / d (rho, vp, vs).

All arithmetic runs in the CUDA library; this file only wires it into
torch.autograd.  The scaling by the incoming gradient of the scalar output
is the autograd contract (one scalar multiply per parameter map).
"""
from __future__ import annotations

import torch

from . import Mesh


class FwiMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, vp, vs, mesh: Mesh, shot_ids, d_obs, ckpt_every: int = 400):
        for t in (rho, vp, vs, d_obs):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise TypeError("FwiMisfit expects contiguous float32 CUDA tensors")
        mesh.set_model(rho, vp, vs)
        f = mesh.misfit(shot_ids, d_obs)
        ctx.mesh, ctx.shot_ids, ctx.ckpt = mesh, list(shot_ids), int(ckpt_every)
        ctx.save_for_backward(rho, vp, vs, d_obs)
        return torch.tensor(f, dtype=torch.float64, device=rho.device)

    @staticmethod
    def backward(ctx, gout):
        rho, vp, vs, d_obs = ctx.saved_tensors
        mesh = ctx.mesh
        mesh.set_model(rho, vp, vs)
        grad = torch.empty(3, *rho.shape, dtype=torch.float32, device=rho.device)
        mesh.adjoint_gradient(ctx.shot_ids, d_obs, grad, ctx.ckpt)
        s = gout.to(torch.float32)
        return grad[0] * s, grad[1] * s, grad[2] * s, None, None, None, None


def fwi_misfit(rho, vp, vs, mesh: Mesh, shot_ids, d_obs, ckpt_every: int = 400):
    """Misfit (FP64 scalar tensor) of the model (rho, vp, vs) [nz][nx]."""
    return FwiMisfit.apply(rho, vp, vs, mesh, shot_ids, d_obs, ckpt_every)
