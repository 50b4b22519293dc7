"""Fit of material parameters (barrier Ea and field coupling kappa) to
learning/forgetting curves of many devices, by gradient descent on the
likelihood-ratio gradient.

The curve of a device is its conductance G(t) = Zc_t[0] / N, the fraction of
its N ions in the first zone (the first decile at Z = 10), sampled at given
steps.  Each iteration advances all devices together in the batch's
persistent launches (one per tile shape) at the current (Ea, kappa), and the
loss

    loss = sum over devices d, samples k of (G_d(t_k) - G*_d(t_k))^2

has the gradient sum_{d,k} 2 (G_d(t_k) - G*_d(t_k)) dE[G_d(t_k)]/d theta, whose
expectations come from the devices' backward passes, run together in the
batched gradient launches (kmc_batch_grad_all), with the weights 2 (G - G*) / N on the
zone-0 counts.  The sampled G replaces its
expectation in the factor 2 (G - G*), which is exact as the devices' rail
counts grow (G's own variance is O(1 / ions)).
"""
from __future__ import annotations

import dataclasses
import time
from typing import List, Optional

import numpy as np

from . import kmc as K


@dataclasses.dataclass
class FitStep:
    Ea: float
    kappa: float
    loss: float
    grad: np.ndarray          # dloss / d(Ea, kappa)
    stderr: np.ndarray        # standard error of grad
    seconds_forward: float
    seconds_backward: float


class MaterialFit:
    """Devices, their protocol and target curves; evaluates loss and gradient."""

    def __init__(self, devs, V: np.ndarray, fills, sample_steps: np.ndarray, target: np.ndarray,
                 warps: int = 8, steps_per_launch: int = 1024, stream: Optional[int] = None):
        self.devs = list(devs)
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.fills = list(fills)
        self.sample_steps = np.asarray(sample_steps, dtype=np.int64)
        self.target = np.asarray(target, dtype=np.float64)
        if self.target.shape != (len(self.devs), len(self.sample_steps)):
            raise ValueError("target must be [devices, samples]")
        self.n_steps = int(self.sample_steps.max()) + 1
        self.warps, self.steps_per_launch = warps, steps_per_launch
        self.stream = stream

    def loss(self, Ea: float, kappa: float):
        """(loss, curves G [devices, samples], forward seconds) at (Ea, kappa),
        without the backward pass."""
        import torch
        devs = [dataclasses.replace(d, Ea=Ea, kappa=kappa) for d in self.devs]
        n = len(devs)
        b = K.Batch(devs, [self.V] * n, [1] * n, fills=self.fills, stream=self.stream)
        try:
            b.set_launch(self.warps, self.steps_per_launch)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step_n(self.n_steps)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            G = np.zeros_like(self.target)
            for i in range(n):
                _, Zc = b.traces(i)
                G[i] = Zc[self.sample_steps, 0] / max(float(Zc[0].sum()), 1.0)
        finally:
            b.close()
        return float(((G - self.target) ** 2).sum()), G, t1 - t0

    def loss_and_grad(self, Ea: float, kappa: float) -> FitStep:
        import torch
        devs = [dataclasses.replace(d, Ea=Ea, kappa=kappa) for d in self.devs]
        n = len(devs)
        b = K.Batch(devs, [self.V] * n, [1] * n, fills=self.fills, stream=self.stream)
        try:
            b.set_launch(self.warps, self.steps_per_launch)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.step_n(self.n_steps)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            G = np.zeros_like(self.target)
            N = np.zeros(n)
            for i in range(n):
                _, Zc = b.traces(i)
                N[i] = max(float(Zc[0].sum()), 1.0)       # ions (conserved: blocking)
                G[i] = Zc[self.sample_steps, 0] / N[i]
            r = G - self.target
            loss = float((r ** 2).sum())
            wZs = []
            for i in range(n):
                wZ = np.zeros((self.n_steps, devs[i].Z))
                wZ[self.sample_steps, 0] = 2.0 * r[i] / N[i]
                wZs.append(wZ)
            # every device's backward pass in one batched launch
            g, se = b.grad_all(None, wZs)
            grad = g[:, [0, 2]].sum(axis=0)
            var = (se[:, [0, 2]] ** 2).sum(axis=0)
            t2 = time.perf_counter()
        finally:
            b.close()
        return FitStep(Ea, kappa, loss, grad, np.sqrt(var), t1 - t0, t2 - t1)

    def run(self, Ea0: float, kappa0: float, iters: int, lr=(6e-3, 5e-2),
            betas=(0.8, 0.95)) -> List[FitStep]:
        """Adam on (Ea, kappa) with per-parameter step sizes lr (eV, 1); the
        last entry is the evaluation at the final parameters."""
        theta = np.array([Ea0, kappa0], dtype=np.float64)
        m = np.zeros(2)
        v = np.zeros(2)
        lr = np.asarray(lr, dtype=np.float64)
        hist = []
        for it in range(1, iters + 1):
            st = self.loss_and_grad(float(theta[0]), float(theta[1]))
            hist.append(st)
            m = betas[0] * m + (1 - betas[0]) * st.grad
            v = betas[1] * v + (1 - betas[1]) * st.grad ** 2
            mh = m / (1 - betas[0] ** it)
            vh = v / (1 - betas[1] ** it)
            theta = theta - lr * mh / (np.sqrt(vh) + 1e-30)
        hist.append(self.loss_and_grad(float(theta[0]), float(theta[1])))
        return hist
