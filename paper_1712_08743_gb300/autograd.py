"""torch.autograd.Function for the FWI misfit of Eq. 4 with a hand-written backward.

``HelmFWI.apply(m, problem)`` returns J(m) as a 0-d float64 tensor. Its forward
runs the batched forward solves (helm_fwi_forward) and keeps the wavefields on
the device; its backward runs the adjoint Helmholtz solves with B^H and forms
dJ/dm (helm_fwi_backward, Eq. 7) in the library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import api


@dataclass
class FWIProblem:
    ctx: api.Context
    h: float
    omegas: np.ndarray          # [nf] angular frequencies
    src: np.ndarray             # [ns, 2] physical (ix, iz)
    rec: np.ndarray             # [nr, 2] physical (ix, iz)
    d_obs: np.ndarray           # [nf][ns][nr] complex128
    lam: float = 0.0            # regulariser weight of Eq. 4
    npml: int = 20
    alpha_max: float = 0.5
    opts: dict = field(default_factory=dict)


class HelmFWI(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m: torch.Tensor, problem: FWIProblem):
        slow = m.detach().to("cpu", torch.float64).contiguous().numpy()
        model = api.helm_create_model(problem.ctx, slow, problem.h, problem.npml, problem.alpha_max)
        J, d_cal, state, stats, status = api.helm_fwi_forward(model, problem.omegas, problem.src, problem.rec,
                                                               problem.d_obs, problem.lam, problem.opts)
        ctx.model, ctx.state, ctx.problem = model, state, problem
        ctx.fwd_stats = stats
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, grad_J):
        g, status = api.helm_fwi_backward(ctx.model, ctx.state, ctx.problem.opts)
        ctx.state.close()
        ctx.model.close()
        grad = torch.from_numpy(g).to(grad_J.device)
        return grad_J * grad, None
