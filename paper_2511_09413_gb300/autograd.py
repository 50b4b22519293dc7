"""torch.autograd front end of the likelihood-ratio gradient (kmc_grad).

``simulate(theta, dev, V, n_steps)`` runs one device on the GPU for n_steps
with theta = (Ea, nu, kappa, fill) and returns its traces (J [n], Zc [n, Z])
as float64 tensors.  The stochastic dynamics are not changed: the traces are
integer counts and carry no pathwise derivative.  Backward contracts the
incoming gradient with the likelihood-ratio estimate of d E[traces] / d theta,
computed by the CUDA backward pass, which replays the trajectory from its
initial occupancy and accumulates the score in FP64.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np
import torch

from . import kmc as K


class KmcTraces(torch.autograd.Function):
    """(J, Zc) of one simulated device as a function of (Ea, nu, kappa, fill)."""

    @staticmethod
    def forward(ctx, theta, dev, V, n_steps, init_mode, occ0):
        Ea, nu, kappa, fill = (float(x) for x in theta.detach().cpu().tolist())
        d = dataclasses.replace(dev, Ea=Ea, nu=nu, kappa=kappa)
        sim = K.Sim(d, V, init_mode, fill=fill, occ0=occ0)
        sim.step_n(int(n_steps))
        J, Zc = sim.traces()
        ctx.sim = sim
        ctx.bernoulli = init_mode == 1
        return torch.from_numpy(J.astype(np.float64)), torch.from_numpy(Zc.astype(np.float64))

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gJ, gZc):
        sim = ctx.sim
        wJ = gJ.detach().cpu().double().numpy()
        wZ = gZc.detach().cpu().double().numpy()
        g, se = sim.grad(wJ if np.any(wJ) else None, wZ if np.any(wZ) else None)
        sim.close()
        ctx.sim = None
        if not ctx.bernoulli:
            g[3] = 0.0      # the placement does not depend on fill
        ctx.stderr = se
        return torch.from_numpy(g), None, None, None, None, None


def simulate(theta: torch.Tensor, dev, V: np.ndarray, n_steps: int, init_mode: int = 1,
             occ0: Optional[np.ndarray] = None):
    """Traces (J, Zc) of ``dev`` with (Ea, nu, kappa, fill) = theta (float64,
    4 entries); differentiable with respect to theta in expectation."""
    if theta.shape != (4,):
        raise ValueError("theta must hold (Ea, nu, kappa, fill)")
    return KmcTraces.apply(theta.to(torch.float64), dev, V, n_steps, init_mode, occ0)
