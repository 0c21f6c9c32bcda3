"""torch.autograd bindings of the forward run and its discrete adjoint.

``BMERun.apply(W0, grid, nsteps, K)`` advances the primitive initial state ``W0`` (a CUDA
tensor [10][nz][ny][nx] in the grid's precision) by ``nsteps`` CFL steps on ``grid`` and
returns the conserved final state.  The forward run records the adjoint tape
(``msh_set_tape``: checkpoints every ``K`` steps written by the step kernels, the dt of
every step, which steps tagged fallback cells); ``backward`` calls ``msh_adjoint_tape``
(dt schedule, limiter and fallback branches frozen; segments recomputed from the
checkpoints) and returns dL/dW0.  Everything runs in libmsh; torch only holds the buffers
and chains the gradient into whatever produced W0 and whatever consumes U_N.  A later
``set_state`` or ``set_time`` on the grid ends the recording, so ``backward`` must run
before the grid is reused.
"""
from __future__ import annotations

import torch

from . import msh


class BMERun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, W0, grid, nsteps, K):
        W0 = W0.detach().contiguous()
        grid.set_time(0.0, 0)
        grid.set_state(W0, msh.PRIMITIVE)
        grid.set_recording(int(nsteps))
        grid.set_tape(int(K), int(nsteps))
        steps, _ = grid.run(max_steps=int(nsteps))
        if steps != nsteps:
            raise RuntimeError(f"forward run stopped after {steps} of {nsteps} steps")
        UN = torch.empty_like(W0)
        grid.get_state(msh.CONSERVED, out=UN)
        ctx.grid = grid
        return UN

    @staticmethod
    def backward(ctx, gUN):
        g = ctx.grid
        want = torch.float32 if g.precision == msh.FP32 else torch.float64
        gW0 = g.adjoint_tape(gUN.contiguous().to(want), kind=msh.PRIMITIVE)
        return gW0, None, None, None


def run(W0, grid, nsteps, K=50):
    """Differentiable forward run (see BMERun)."""
    return BMERun.apply(W0, grid, nsteps, K)
