"""Differentiable stellar-disc workload: gradient of the m = 2 spiral amplitude with respect
to the initial density perturbation and the dispersion anisotropy.

The loss is the global Fourier amplitude of Sec. 4.4,
    A_m = | sum_{R < R_loss} Sigma e^{i m phi} dA | / M_d,   m = 2,
at the final time, with M_d the total disc mass on the grid.  The initial state is the
disc of ``inputs.disc`` composed in torch from (delta, beta), so autograd chains
dL/dW0 (from ``msh_adjoint_run``) into dL/d delta and dL/d beta.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import autograd, inputs, msh


def fourier_amplitude(UN, base, m=2, R_loss=10.0):
    """A_m of the surface density (component 0 of the conserved state)."""
    Sig = UN[0, 0].to(torch.float64)
    dev = Sig.device
    X = torch.as_tensor(base["X"], device=dev)
    Y = torch.as_tensor(base["Y"], device=dev)
    R = torch.as_tensor(base["R"], device=dev)
    dA = base["dx"] * base["dx"]
    ph = torch.atan2(Y, X)
    w = (R < R_loss).to(torch.float64) * dA
    re = (Sig * torch.cos(m * ph) * w).sum()
    im = (Sig * torch.sin(m * ph) * w).sum()
    Md = Sig.sum() * dA
    return torch.sqrt(re * re + im * im) / Md


class DiscProblem:
    """The disc on an n x n grid with a fixed step count, precision and checkpoint interval."""

    def __init__(self, n=512, nsteps=2000, precision=msh.FP32, K=50, seed=5, stream=None):
        p = inputs.disc(n=n, nsteps=nsteps, seed=seed)
        self.problem = p
        self.base = inputs.disc_base(n)
        self.nsteps, self.K = nsteps, K
        self.dtype = torch.float32 if precision == msh.FP32 else torch.float64
        self.grid = msh.Grid.from_problem(p, precision, stream=stream)
        self.delta0 = torch.tensor(0.01 * inputs.disc_noise(n, seed), dtype=torch.float64, device="cuda")
        self.tbase = {k: (torch.as_tensor(v, device="cuda") if isinstance(v, np.ndarray) else v)
                      for k, v in self.base.items()}

    def initial_state(self, delta, beta):
        return inputs.disc_compose(self.tbase, delta, beta, xp=torch)

    def loss(self, delta, beta):
        W0 = self.initial_state(delta, beta).to(self.dtype).contiguous()
        UN = autograd.run(W0, self.grid, self.nsteps, self.K)
        return fourier_amplitude(UN, self.base, 2, self.problem.extra["R_loss"])

    def value_and_grad(self, delta=None, beta=0.0):
        delta = (self.delta0 if delta is None else delta).clone().requires_grad_(True)
        beta = torch.tensor(float(beta), dtype=torch.float64, device="cuda", requires_grad=True)
        L = self.loss(delta, beta)
        gd, gb = torch.autograd.grad(L, (delta, beta))
        return float(L.detach()), gd, float(gb)

    def close(self):
        self.grid.close()
