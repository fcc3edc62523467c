"""torch.autograd.Function over lbm_adjoint_step: a scalar objective of a
simulation as a function of body-kinematics parameters theta, with the
gradient from the hand-written adjoint (no tape)."""
from __future__ import annotations

import numpy as np
import torch


class KinematicsObjective(torch.autograd.Function):
    """J(theta) with dJ/dtheta from one forward + adjoint run.  ``run`` maps a
    numpy theta to (J, dJ/dtheta) (see kinematics_objective)."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, run):
        J, dJ = run(theta.detach().cpu().numpy().astype(np.float64))
        ctx.save_for_backward(torch.as_tensor(np.asarray(dJ), dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad):
        (dJ,) = ctx.saved_tensors
        return grad * dJ, None


def kinematics_objective(make_lattice, horizon: int, w_force, checkpoint_every: int = 0):
    """Returns f(theta) -> J as a differentiable torch function.
    make_lattice(theta) must return a Lattice at its initial state with a
    swimmer (held, or free in any of x, y and yaw) whose (wave_amp,
    wave_length, wave_period) are theta; J is the mean of w_force . F over
    ``horizon`` steps (w_force = e_swim for the thrust)."""

    def run(theta):
        lat = make_lattice(theta)
        try:
            out = lat.adjoint(horizon, w_force, checkpoint_every=checkpoint_every)
        finally:
            lat.close()
        return out["J"], out["dJ_dtheta"]

    def f(theta: torch.Tensor) -> torch.Tensor:
        return KinematicsObjective.apply(theta, run)

    return f
