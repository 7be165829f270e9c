"""Differentiation through the engine: U(x, lambda, theta) as a
torch.autograd.Function whose backward is the engine's hand-written
derivative pass.

theta = (epsilon, sigma, q) of every alchemical atom.  forward() hands the
CUDA tensors x, lambda and theta to la_energy_forces_device, which replaces
the walker's positions, lambda and the system's alchemical parameters on the
device, rebuilds the walker's neighbour lists from x (recomputation instead
of storage) and evaluates U; the same pass writes -dU/dx (forces),
dU/dlambda and dU/dtheta into device tensors, which backward() scales by the
incoming gradient.  Nothing passes through host memory and no call
synchronises.  The arithmetic is entirely in the CUDA library; this module
only moves tensors.  The paper does not differentiate with respect to
force-field parameters; gradients of U and of Delta A with respect to the
solute's parameters are an extension of this library.
"""
from __future__ import annotations

import numpy as np
import torch

from .labf import LA_N_TERMS, Engine


class LambdaABFEnergy(torch.autograd.Function):
    """U = LambdaABFEnergy.apply(x, lam, theta, engine, walker).

    x: (n, 3) positions on the engine's device; lam: 0-d tensor; theta:
    (n_alch, 3) tensor of (epsilon, sigma, q).  Returns a 0-d float64 tensor
    on x's device.  Gradients: x -> dU/dx, lam -> dU/dlambda,
    theta -> dU/dtheta.  The forces are written only when x needs a gradient.
    """

    @staticmethod
    def forward(ctx, x, lam, theta, engine: Engine, walker: int):
        dev = engine.device
        n_alch = theta.shape[0]
        P = 3 * n_alch + 1
        xd = x.detach().to(device=dev, dtype=torch.float32).contiguous()
        th = theta.detach().to(device=dev, dtype=torch.float64).contiguous()
        ld = torch.as_tensor(lam, dtype=torch.float64).detach().to(dev).reshape(1).contiguous()
        out = torch.empty(LA_N_TERMS + 2 + 2 * P, dtype=torch.float64, device=dev)
        F = torch.empty((xd.shape[0], 3), dtype=torch.float32, device=dev) if ctx.needs_input_grad[0] else None
        engine.energy_forces_device(walker, x=xd, theta=th, lam=ld, out=out, forces=F)
        dudl = out[LA_N_TERMS + 1]
        dth = out[LA_N_TERMS + 2:LA_N_TERMS + 2 + 3 * n_alch].reshape(n_alch, 3)
        ctx.save_for_backward(F if F is not None else torch.empty(0, device=dev), dudl, dth)
        ctx.x_meta = (x.device, x.dtype)
        ctx.lam_meta = (lam.device, lam.dtype) if torch.is_tensor(lam) else (dev, torch.float64)
        ctx.th_meta = (theta.device, theta.dtype)
        return out[LA_N_TERMS].to(x.device)

    @staticmethod
    def backward(ctx, g):
        F, dudl, dth = ctx.saved_tensors
        gx = gl = gt = None
        if ctx.needs_input_grad[0]:
            gx = (-F.to(torch.float64) * g.to(F.device)).to(*ctx.x_meta)
        if ctx.needs_input_grad[1]:
            gl = (dudl * g.to(dudl.device)).to(*ctx.lam_meta)
        if ctx.needs_input_grad[2]:
            gt = (dth * g.to(dth.device)).to(*ctx.th_meta)
        return gx, gl, gt, None, None


def energy(engine: Engine, walker: int, x, lam, theta):
    return LambdaABFEnergy.apply(x, lam, theta, engine, walker)


def theta_of(spec) -> np.ndarray:
    """(n_alch, 3) array of (epsilon, sigma, q) of the alchemical atoms."""
    idx = np.nonzero(spec.alch)[0]
    return np.stack([spec.epsilon[idx], spec.sigma[idx], spec.charge[idx]], axis=1)
