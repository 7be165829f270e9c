"""Differentiation through the engine: U(x, lambda, theta) as a
torch.autograd.Function whose backward is the engine's hand-written
derivative pass.

theta = (epsilon, sigma, q) of every alchemical atom.  forward() uploads the
configuration, rebuilds the neighbour lists for it (recomputation instead of
storage) and evaluates U; the same engine call also returns -dU/dx (forces),
dU/dlambda and dU/dtheta, which backward() scales by the incoming gradient.
The arithmetic is entirely in the CUDA library; this module only moves
tensors.  The paper does not differentiate with respect to force-field
parameters; gradients of U and of Delta A with respect to the solute's
parameters are an extension of this library.
"""
from __future__ import annotations

import numpy as np
import torch

from .labf import Engine


class LambdaABFEnergy(torch.autograd.Function):
    """U = LambdaABFEnergy.apply(x, lam, theta, engine, walker).

    x: (n, 3) positions (any device, float); lam: 0-d tensor; theta:
    (n_alch, 3) tensor of (epsilon, sigma, q).  Returns a 0-d float64 tensor on
    x's device.  Gradients: x -> dU/dx, lam -> dU/dlambda, theta -> dU/dtheta.
    """

    @staticmethod
    def forward(ctx, x, lam, theta, engine: Engine, walker: int):
        sys = engine.walker_sys[walker]
        engine.set_alch_params(sys, theta.detach().to("cpu", torch.float64).numpy())
        engine.set_state(walker, x=x.detach().to("cpu", torch.float32).numpy(), lam=float(lam))
        r = engine.energy_forces(walker)
        n_alch = theta.shape[0]
        ctx.save_for_backward(r["F"].to(x.device, x.dtype),
                              torch.tensor(r["dUdl"], dtype=torch.float64, device=x.device),
                              torch.tensor(r["dth"][:3 * n_alch].reshape(n_alch, 3), dtype=theta.dtype,
                                           device=theta.device))
        ctx.lam_dtype = lam.dtype if torch.is_tensor(lam) else torch.float64
        return torch.tensor(r["U"], dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, g):
        F, dudl, dth = ctx.saved_tensors
        gx = -F * g.to(F.dtype)
        gl = (dudl * g).to(ctx.lam_dtype)
        gt = dth * g.to(dth.dtype)
        return gx, gl, gt, None, None


def energy(engine: Engine, walker: int, x, lam, theta):
    return LambdaABFEnergy.apply(x, lam, theta, engine, walker)


def theta_of(spec) -> np.ndarray:
    """(n_alch, 3) array of (epsilon, sigma, q) of the alchemical atoms."""
    idx = np.nonzero(spec.alch)[0]
    return np.stack([spec.epsilon[idx], spec.sigma[idx], spec.charge[idx]], axis=1)
