"""torch.autograd bindings of the forward run and its discrete adjoint.

``BMERun.apply(W0, grid, nsteps, K)`` advances the primitive initial state ``W0`` (a CUDA
tensor [10][nz][ny][nx] in the grid's precision) by ``nsteps`` CFL steps on ``grid`` and
returns the conserved final state.  The dt schedule of the forward run is recorded and
frozen; ``backward`` calls ``msh_adjoint_run`` (checkpoints every ``K`` steps, limiter and
fallback branches frozen) and returns dL/dW0.  Everything runs in libmsh; torch only holds
the buffers and chains the gradient into whatever produced W0 and whatever consumes U_N.
"""
from __future__ import annotations

import numpy as np
import torch

from . import msh


class BMERun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W0, grid, nsteps, K):
        W0 = W0.detach().contiguous()
        grid.set_time(0.0, 0)
        grid.set_state(W0, msh.PRIMITIVE)
        grid.set_recording(int(nsteps))
        steps, _ = grid.run(max_steps=int(nsteps))
        if steps != nsteps:
            raise RuntimeError(f"forward run stopped after {steps} of {nsteps} steps")
        dts = grid.dt_history()
        UN = torch.empty_like(W0)
        grid.get_state(msh.CONSERVED, out=UN)
        ctx.save_for_backward(W0)
        ctx.grid, ctx.dts, ctx.K = grid, np.array(dts), int(K)
        return UN

    @staticmethod
    def backward(ctx, gUN):
        (W0,) = ctx.saved_tensors
        gW0 = ctx.grid.adjoint_run(W0, ctx.dts, gUN.contiguous().to(W0.dtype), K=ctx.K, kind=msh.PRIMITIVE)
        return gW0, None, None, None


def run(W0, grid, nsteps, K=50):
    """Differentiable forward run (see BMERun)."""
    return BMERun.apply(W0, grid, nsteps, K)
