"""Fit probe radiance to captured views (the differentiable-fit workload).

The forward pass is the tracer (lfp_render_ex) and the backward pass the
adjoint kernel (lfp_render_backward_ex), joined by the torch.autograd.Function
in this package; the optimiser is torch's fused Adam over the radiance
tensor. Distance and normal maps stay fixed, so the loss is quadratic in
radiance and Adam converges to the noise floor of the targets.

Data parallel: with a process group of W ranks, rank r renders views r, r+W,
... and scatters its pixels' gradients locally; one all-reduce (sum) of the
radiance gradient per step then gives every rank the gradient of the whole
loss, and the replicated Adam steps stay identical.

Checkpoint / resume: with `checkpoint=path`, the radiance, the Adam state,
the step and the history are saved every `checkpoint_every` steps and after
the last (torch.save to a temporary file, then an atomic rename; rank 0 of a
group writes, the ranks hold identical state), and a fit that finds the file
continues after its step.
"""
from __future__ import annotations

import os
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


def shard_views(views, rank: int, world: int):
    """The views rank `rank` of `world` renders: every world-th, from `rank`."""
    return list(views)[rank::world]


def shard_pixels(views, rank: int, world: int):
    """Flat pixel index ranges ([begin, end) into the concatenated views) of
    the rank's views, in its rendering order."""
    offs, o = [], 0
    for v in views:
        offs.append((o, o + v.W * v.H))
        o += v.W * v.H
    return offs[rank::world]


def allreduce_gradient(grad, group=None):
    """Sum a gradient over the ranks of `group` (no-op without one)."""
    import torch.distributed as dist
    if group is not None or (dist.is_available() and dist.is_initialized()):
        if dist.get_world_size(group) > 1:
            dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad


def _rank(group):
    import torch.distributed as dist
    return dist.get_rank(group) if dist.is_available() and dist.is_initialized() else 0


def save_checkpoint(path: str, step: int, rad, opt, history, group=None) -> None:
    """Atomically write the fit state after `step` (rank 0 only)."""
    if _rank(group) != 0:
        return
    tmp = f"{path}.tmp"
    torch.save({"step": step, "radiance": rad.detach(), "adam": opt.state_dict(), "history": list(history)}, tmp)
    os.replace(tmp, path)


def fit_radiance(grid: ProbeGrid, views, targets, steps: int = 200, lr: float = 1e-2, seed: int = 404,
                 init=None, log_every: int = 0, group=None, total_pixels=None, checkpoint: str | None = None,
                 checkpoint_every: int = 0):
    """Fit radiance [P][N][N][3] (re-initialised U[0,1] unless `init` is given)
    to `targets` [pixels][3] with an L2 loss (the mean over all ranks' pixels
    and channels). With a process group, `views` / `targets` are this rank's
    shard (shard_views / shard_pixels) and `total_pixels` the pixels of all
    ranks. `checkpoint`: see the module docstring; `steps` counts from the
    start of the fit, resumed or not. Returns (radiance, history) where
    history holds (step, mse, ms) tuples of the logged steps and the last one
    (mse of this rank's shard)."""
    P, N = grid.n_probes, grid.N
    if init is None:
        gen = torch.Generator(device="cuda").manual_seed(seed)
        init = torch.rand((P, N, N, 3), device="cuda", generator=gen)
    rad = init.clone().requires_grad_(True)
    opt = torch.optim.Adam([rad], lr=lr, fused=True)
    denom = 3.0 * (targets.shape[0] if total_pixels is None else total_pixels)
    history = []
    first = 0
    if checkpoint and os.path.exists(checkpoint):
        state = torch.load(checkpoint, map_location=rad.device, weights_only=False)
        with torch.no_grad():
            rad.copy_(state["radiance"])
        opt.load_state_dict(state["adam"])
        history = [tuple(h) for h in state["history"]]
        first = int(state["step"]) + 1
    t0 = time.perf_counter()
    for it in range(first, steps):
        opt.zero_grad(set_to_none=False)
        rgb, _ = render(rad, grid, views)
        loss = ((rgb - targets) ** 2).sum() / denom
        loss.backward()
        allreduce_gradient(rad.grad, group)
        opt.step()
        if (log_every and it % log_every == 0) or it == steps - 1:
            torch.cuda.synchronize()
            mse = ((rgb.detach() - targets) ** 2).mean().item()
            history.append((it, mse, (time.perf_counter() - t0) * 1e3 / (it + 1 - first)))
        if checkpoint and ((checkpoint_every and (it + 1) % checkpoint_every == 0) or it == steps - 1):
            save_checkpoint(checkpoint, it, rad, opt, history, group)
    return rad.detach(), history
