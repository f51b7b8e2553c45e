"""Fit probe radiance to captured views (the differentiable-fit workload).

The forward pass is the tracer (lfp_render_ex) and the backward pass the
adjoint kernel (lfp_render_backward_ex), joined by the torch.autograd.Function
in this package; the optimiser is torch's fused Adam over the radiance
tensor. Distance and normal maps stay fixed, so the loss is quadratic in
radiance and Adam converges to the noise floor of the targets.
"""
from __future__ import annotations

import time

import torch

from . import ProbeGrid, render


def make_targets(grid: ProbeGrid, views, sigma: float = 0.01, seed: int = 404):
    """Render the views with the grid's current radiance and add N(0, sigma^2) noise."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    with torch.no_grad():
        clean = grid.render(views, aux=False)["rgb"]
        noise = torch.randn(clean.shape, device=clean.device, generator=gen) * sigma
    return clean + noise


def fit_radiance(grid: ProbeGrid, views, targets, steps: int = 200, lr: float = 1e-2, seed: int = 404,
                 init=None, log_every: int = 0):
    """Fit radiance [P][N][N][3] (re-initialised U[0,1] unless `init` is given)
    to `targets` [pixels][3] with an L2 loss. Returns (radiance, history) where
    history holds (step, mse, ms) tuples of the logged steps and the last one."""
    P, N = grid.n_probes, grid.N
    if init is None:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        init = torch.rand((P, N, N, 3), device="cuda", generator=gen)
    rad = init.clone().requires_grad_(True)
    opt = torch.optim.Adam([rad], lr=lr, fused=True)
    history = []
    t0 = time.perf_counter()
    for it in range(steps):
        opt.zero_grad(set_to_none=False)
        rgb, _ = render(rad, grid, views)
        loss = ((rgb - targets) ** 2).mean()
        loss.backward()
        opt.step()
        if (log_every and it % log_every == 0) or it == steps - 1:
            torch.cuda.synchronize()
            history.append((it, loss.item(), (time.perf_counter() - t0) * 1e3 / (it + 1)))
    return rad.detach(), history
