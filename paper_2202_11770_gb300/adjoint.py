"""``torch.autograd.Function`` over the solver's discrete adjoint.

``flow_objective(tau, amps, solver, ...)`` returns the objective
``J = (1/N) sum_{t=1..N} sum_p (u(x_p, t).axis - target_p)^2`` of an N-step run
started from equilibrium, as a differentiable function of the relaxation time
``tau`` and of the inlet amplitude groups ``amps`` (all groups of all
velocity iolets, iolet by iolet).  The forward call runs the library's
``hlb_adjoint_run``: N forward steps with sqrt(N)-spaced checkpoints, then the
exact transpose of every step (collision, streaming, bounce-back, Ladd and
pressure boundaries) — so dJ/dtau and dJ/da are available when forward
returns, and backward only scales them by the incoming gradient.

There is no counterpart in arXiv 2202.11770; the adjoint differentiates the
paper's LBGK step (Eqs. 3a-3b, 4-6) with its Section 2.3 boundaries.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hemegb


class FlowObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, tau, amps, solver, nsteps, sites, target, axis, waves, rho0, workspace):
        tau_v = float(tau.detach().cpu())
        a = amps.detach().cpu().double().numpy()
        solver.set_tau(tau_v)
        off = 0
        for k, io in enumerate(solver.iolets):
            if io.kind != hemegb.HLB_VELOCITY:
                continue
            g = int(io.n_groups)
            solver.set_velocity(k, a[off:off + g], waves[k])
            off += g
        if off != a.size:
            raise ValueError(f"expected {off} amplitudes, got {a.size}")
        solver.init_equilibrium(rho0)
        J, dtau, damp = solver.adjoint(nsteps, sites, target, axis, workspace=workspace)
        ctx.save_for_backward(torch.tensor(dtau, dtype=torch.float64),
                              torch.as_tensor(np.asarray(damp), dtype=torch.float64))
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        dtau, damp = ctx.saved_tensors
        g = gJ.to(torch.float64).cpu()
        return (g * dtau, g * damp) + (None,) * 8


def flow_objective(tau, amps, solver, nsteps, sites, target, axis, waves, rho0=1.0, workspace=None):
    """Differentiable objective of an N-step run from equilibrium rho0.

    tau: 0-d float64 tensor; amps: 1-d float64 tensor with one entry per
    amplitude group of every velocity iolet (iolet order); waves: dict
    iolet -> waveform (as for Solver.set_velocity); sites/target/axis: the
    probe sites, their target axial velocities and the axis."""
    return FlowObjective.apply(tau, amps, solver, nsteps, sites, target, axis, waves, rho0, workspace)
