"""torch.autograd bridge to the hand-written adjoint (nlc_adjoint).

`droplet_loss(Q0, params, ...)` runs the droplet problem forward on the GPU
from the initial order-parameter field Q0 and returns the loss
L = w_R (R - R_target)^2 + w_u |u|_2 of the final state as a torch scalar
that is differentiable with respect to Q0 and to the (gamma, K, Gamma)
entries of `params`.  The forward pass already runs the adjoint (its forward
sweep is the forward run), so backward only scales the stored gradients.
"""
import numpy as np
import torch

from . import nlc


class DropletLoss(torch.autograd.Function):
    """forward(Q0 [5,nz,ny,nx], theta [gamma, K, Gamma], sim, nsteps,
    ckpt_every, target_radius, w_radius, w_velocity) -> L"""

    @staticmethod
    def forward(ctx, Q0, theta, sim, base_params, nsteps, ckpt_every,
                target_radius, w_radius, w_velocity):
        p = dict(base_params)
        p["gamma"], p["K"], p["Gamma"] = (float(v) for v in theta.detach().cpu())
        sim.set_params(p)
        sim.set_fields(Q0.detach().to("cpu", torch.float64).numpy())
        g = sim.adjoint(target_radius, w_radius, w_velocity, nsteps=nsteps,
                        ckpt_every=ckpt_every, want_dQ0=True)
        ctx.save_for_backward(
            torch.from_numpy(np.ascontiguousarray(g["dQ0"])).to(Q0),
            torch.tensor([g["dgamma"], g["dK"], g["dGamma"]], dtype=theta.dtype,
                         device=theta.device))
        return torch.tensor(g["loss"], dtype=Q0.dtype, device=Q0.device)

    @staticmethod
    def backward(ctx, grad_out):
        dQ0, dtheta = ctx.saved_tensors
        return (grad_out * dQ0, grad_out * dtheta, None, None, None, None, None,
                None, None)


def droplet_loss(Q0, theta, sim, base_params, nsteps, ckpt_every,
                 target_radius, w_radius=1.0, w_velocity=1.0):
    """Differentiable loss of the droplet problem (see module docstring)."""
    return DropletLoss.apply(Q0, theta, sim, base_params, nsteps, ckpt_every,
                             target_radius, w_radius, w_velocity)
