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
from torch.autograd.function import once_differentiable

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
    """J(m) with one backward: the forward keeps the wavefields and data residuals on
    the device (a library FwiState), the backward consumes them with the adjoint
    solves and releases them. A second backward through the same graph raises; a
    forward whose graph is dropped without a backward frees its state when the
    autograd context is collected (FwiState and Model close themselves)."""

    @staticmethod
    def forward(ctx, m: torch.Tensor, problem: FWIProblem):
        # the model build (padding, multigrid hierarchy, Galerkin operators) runs on the device
        # from a host copy of the physical slowness, which helm_create_model validates
        slow = m.detach().to("cpu", torch.float64).contiguous().numpy()
        model = api.helm_create_model(problem.ctx, slow, problem.h, problem.npml, problem.alpha_max)
        J, d_cal, state, stats, status = api.helm_fwi_forward(model, problem.omegas, problem.src, problem.rec,
                                                               problem.d_obs, problem.lam, problem.opts)
        ctx.model, ctx.state, ctx.problem = model, state, problem
        ctx.fwd_stats = stats
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    @once_differentiable
    def backward(ctx, grad_J):
        if ctx.state is None:
            raise RuntimeError("HelmFWI: backward ran already; its device state was released "
                               "(call forward again for another gradient)")
        if grad_J.is_cuda:
            # the library writes the gradient straight into a device tensor (device_ptrs)
            g = torch.empty((ctx.model.Pz, ctx.model.Px), dtype=torch.float64, device=grad_J.device)
            api.helm_fwi_backward(ctx.model, ctx.state, ctx.problem.opts, grad_out=g)
        else:
            g = torch.from_numpy(api.helm_fwi_backward(ctx.model, ctx.state, ctx.problem.opts)[0])
        ctx.state.close()
        ctx.model.close()
        ctx.state = None
        return grad_J * g, None
