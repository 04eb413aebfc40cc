"""Differentiable implicit time stepping: U_T = Phi(U_0, theta) as a
torch.autograd.Function over the library's SDIRK step and its discrete adjoint.

theta = (d1, d2, gamma, alpha1, alpha2, f1, k_ox, beta1): the reaction
coefficients of Eq. (1) and the immune-cell inflow rate of Eq. (3).  The
forward pass stores U every `checkpoint` steps; the backward pass walks the
segments from last to first, recomputes each segment's steps storing their
stage values (cdg2_step_stages), then applies cdg2_step_adjoint backwards
through the segment.  Host orchestration only: every solve, JVP and VJP
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import torch

from . import (Mesh, SolverOpts, cdg2_step, cdg2_step_adjoint, cdg2_step_stages, make_opts, make_params,
               stages_of)

THETA_NAMES = ("d1", "d2", "gamma", "alpha1", "alpha2", "f1", "k_ox", "beta1")


def _params_with(base: dict, theta: torch.Tensor):
    p = dict(base)
    for i, name in enumerate(THETA_NAMES):
        p[name] = float(theta[i])
    return make_params(p)


class Cdg2Steps(torch.autograd.Function):
    """(U0, theta) -> U after `nsteps` SDIRK steps of size dt from t0."""

    @staticmethod
    def forward(ctx, U0: torch.Tensor, theta: torch.Tensor, mesh: Mesh, base_params: dict, t0: float, dt: float,
                nsteps: int, checkpoint: int, opts: SolverOpts):
        p = _params_with(base_params, theta)
        U = U0.detach().clone().contiguous()
        checkpoints = {}
        for n in range(nsteps):
            if n % checkpoint == 0:
                checkpoints[n] = U.clone()
            cdg2_step(mesh, p, U, t0 + n * dt, dt, opts)
        ctx.mesh, ctx.p, ctx.t0, ctx.dt, ctx.nsteps, ctx.checkpoint, ctx.opts = mesh, p, t0, dt, nsteps, checkpoint, opts
        ctx.checkpoints = checkpoints
        return U

    @staticmethod
    def backward(ctx, gU: torch.Tensor):
        mesh, p, t0, dt, opts = ctx.mesh, ctx.p, ctx.t0, ctx.dt, ctx.opts
        s = stages_of(opts)
        lam = gU.detach().to(torch.float64).clone().contiguous()
        gtheta = torch.zeros(8, dtype=torch.float64, device=lam.device)
        starts = sorted(ctx.checkpoints)
        for k in reversed(range(len(starts))):
            n0 = starts[k]
            n1 = starts[k + 1] if k + 1 < len(starts) else ctx.nsteps
            U = ctx.checkpoints[n0].clone()
            stages = torch.empty((n1 - n0, s * mesh.n_dof), dtype=torch.float64, device=lam.device)
            for n in range(n0, n1):
                cdg2_step_stages(mesh, p, U, t0 + n * dt, dt, stages[n - n0], opts)
            for n in reversed(range(n0, n1)):
                cdg2_step_adjoint(mesh, p, stages[n - n0], t0 + n * dt, dt, lam, gtheta, opts)
        return lam, gtheta, None, None, None, None, None, None, None


def steps(U0: torch.Tensor, theta: torch.Tensor, mesh: Mesh, base_params: dict, t0: float, dt: float, nsteps: int,
          checkpoint: int = 10, opts: SolverOpts = None) -> torch.Tensor:
    """Differentiable U_T; theta is a float64 tensor of the 8 coefficients in THETA_NAMES order."""
    return Cdg2Steps.apply(U0, theta, mesh, base_params, t0, dt, nsteps, max(1, checkpoint), opts or make_opts())
