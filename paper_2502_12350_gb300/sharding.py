"""Shot sharding across ranks (one GPU per rank).

Shots are independent (Algorithm 3 distributes them over MPI ranks with a
static or work-stealing scheduler and ends with two Allreduce calls, misfit
and gradient).  Here shots are partitioned statically by cost (largest
first onto the least-loaded rank, ties to the lower rank), each rank computes
its shard's misfit and gradient through mamute_gradient, and the per-rank
results are summed in ascending rank order on every rank (an all-gather
followed by an ordered sum), so the result is identical on all ranks and
does not depend on the collective's internal reduction order.
"""
from __future__ import annotations

import numpy as np


def partition(costs, world: int):
    """Static cost-balanced partition: list of shot indices per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def shot_costs(grid_nx, grid_ny, grid_nz, border, n_src, aperture=None):
    """Padded points of each shot's propagation domain."""
    Nz = grid_nz + 2 * border
    if aperture is None:
        return [float((grid_nx + 2 * border) * (grid_ny + 2 * border) * Nz)] * n_src
    ap = np.asarray(aperture)
    return [float((a[1] - a[0] + 2 * border) * (a[3] - a[2] + 2 * border) * Nz) for a in ap]


def subset(idx, src_xyz, rec_offset, rec_xyz, aperture=None):
    """Acquisition arrays of the shots idx (receiver offsets rebased) and the
    receiver rows they own in the full data array."""
    src_xyz = np.asarray(src_xyz).reshape(-1, 3)
    rec_xyz = np.asarray(rec_xyz).reshape(-1, 3)
    off = [0]
    rows = []
    for s in idx:
        a, b = int(rec_offset[s]), int(rec_offset[s + 1])
        rows.extend(range(a, b))
        off.append(off[-1] + (b - a))
    ap = None if aperture is None else np.asarray(aperture)[list(idx)]
    return (src_xyz[list(idx)], np.asarray(off, np.int32), rec_xyz[rows] if rows else
            np.zeros((0, 3), np.float32), ap, np.asarray(rows, np.int64))


def ordered_sum(J, grad, group=None):
    """(sum of J, sum of grad) over ranks, added in ascending rank order."""
    import torch
    import torch.distributed as dist
    if group is None and not dist.is_initialized():
        return J, grad
    world = dist.get_world_size(group)
    Jt = torch.tensor([float(J)], dtype=torch.float64, device=grad.device)
    Js = [torch.zeros_like(Jt) for _ in range(world)]
    gs = [torch.zeros_like(grad) for _ in range(world)]
    dist.all_gather(Js, Jt, group=group)
    dist.all_gather(gs, grad.contiguous(), group=group)
    tot = gs[0].clone()
    for r in range(1, world):
        tot += gs[r]
    Jtot = 0.0
    for r in range(world):
        Jtot += float(Js[r].item())
    return Jtot, tot


def sharded_gradient(compute, costs, group=None):
    """Runs compute(shot_indices) -> (J, grad tensor) on this rank's shard and
    returns the ordered sum over ranks."""
    import torch.distributed as dist
    if dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    mine = partition(costs, world)[rank]
    J, grad = compute(mine)
    return ordered_sum(J, grad, group)


def gradient(ctx, grid, vel, rho, src_xyz, wavelet, rec_offset, rec_xyz, d_obs, aperture=None,
             group=None, **opts):
    """Sharded mamute_gradient: each rank handles its shots; every rank
    receives the total misfit and gradient."""
    import torch
    n_src = len(np.asarray(src_xyz).reshape(-1, 3))
    costs = shot_costs(grid.nx, grid.ny, grid.nz, grid.border, n_src, aperture)

    def compute(idx):
        g = torch.zeros_like(vel)
        if not idx:
            return 0.0, g
        src, off, rec, ap, rows = subset(idx, src_xyz, rec_offset, rec_xyz, aperture)
        d = d_obs[torch.as_tensor(rows, device=d_obs.device)].contiguous()
        J = ctx.gradient(grid, vel, rho, src, wavelet, off, rec, d, g, aperture=ap, **opts)
        return J, g

    return sharded_gradient(compute, costs, group)
