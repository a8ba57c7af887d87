"""torch.autograd binding of the differentiation form (u = 0).

``rollout(C0, M, ...)`` advances C0 by nsteps steps of the Cahn-Hilliard
scheme with mobility M = 1/Pe through libch.so; its backward calls the
library's adjoint (ch_step_adjoint), which recomputes the trajectory from
checkpoints, so gradients reach both the initial field and M.
"""
from __future__ import annotations

import torch

from .solver import Solver


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, C0, M, shape, h, bc, cn, dt, nsteps, ckpt_every, precision, w):
        s = Solver(shape, h, bc, cn, 1.0 / float(M), dt, C0.detach(), precision=precision, w=w, device=C0.device)
        s.step(nsteps)
        s.stream.synchronize()
        CT = s.C.clone()
        ctx.solver = s
        ctx.nsteps, ctx.ckpt_every = nsteps, ckpt_every
        ctx.save_for_backward(C0.detach())
        return CT

    @staticmethod
    def backward(ctx, grad_CT):
        (C0,) = ctx.saved_tensors
        s = ctx.solver
        lam0, dM = s.adjoint(C0, ctx.nsteps, grad_CT.contiguous(), ctx.ckpt_every)
        s.stream.synchronize()
        s.close()
        gM = torch.tensor(dM, dtype=torch.float64, device=C0.device)
        return lam0.to(C0.dtype), gM, None, None, None, None, None, None, None, None, None


def rollout(C0, M, shape, h, bc, cn, dt, nsteps, ckpt_every=10, precision="f32", w=4.0):
    """C_T after nsteps steps from C0 (CUDA tensor [nz][ny][nx]); M is a
    0-d tensor (the mobility 1/Pe).  Differentiable in C0 and M."""
    return _Rollout.apply(C0, M, tuple(shape), h, tuple(bc), cn, dt, nsteps, ckpt_every, precision, w)
