"""View sharding of a multi-view training step over ranks (one GPU per rank).

The paper leaves multi-GPU rendering to future work (Sec. 5.3, citing Grendel-style
spatial partitioning).  The natural partition of this path is by camera view: every rank
holds the whole Gaussian set, renders its own views (projection, binning, forward, loss
gradient, backward, projection backward), and one exchange step remains -- the sum over
ranks of the per-Gaussian gradients.  This module holds the host logic of that scheme:

* ``partition_views`` -- which views each rank renders (longest-processing-time-first over
  an estimated per-view load, so ranks finish together);
* ``allreduce_gaussian_grads`` -- the single collective: one flat SUM all-reduce of the
  per-Gaussian gradient tensors (NCCL between GPUs; gloo in the CPU tests);
* ``sharded_gaussian_grads`` -- a rank's step on its views through the library, followed
  by the all-reduce.

Nothing here computes the render path itself; the step calls the C ABI binding.
"""
from __future__ import annotations

import numpy as np
import torch

GRAD_KEYS = ("means3D", "log_scales", "quats", "opacities", "colors")


def partition_views(cams, world: int, loads=None):
    """Views of each rank, longest-processing-time first: views sorted by load (default: the
    pixel count W * H) go one by one to the rank with the least load so far (ties: the lower
    rank).  Returns ``world`` sorted lists of view indices covering every view once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = [float(c["W"] * c["H"]) for c in cams] if loads is None else [float(x) for x in loads]
    if len(w) != len(cams):
        raise ValueError("one load per view")
    order = sorted(range(len(cams)), key=lambda v: (-w[v], v))
    acc = [0.0] * world
    parts = [[] for _ in range(world)]
    for v in order:
        r = min(range(world), key=lambda k: (acc[k], k))
        parts[r].append(v)
        acc[r] += w[v]
    return [sorted(p) for p in parts]


def allreduce_gaussian_grads(grads: dict, group=None, keys=GRAD_KEYS):
    """Sums the per-Gaussian gradient tensors over the ranks of ``group`` in place, with one
    all-reduce of their concatenation (one collective per step).  Returns ``grads``."""
    import torch.distributed as dist
    flat = torch.cat([grads[k].reshape(-1) for k in keys])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k in keys:
        n = grads[k].numel()
        grads[k].copy_(flat[off:off + n].view_as(grads[k]))
        off += n
    return grads


def local_gaussian_grads(plan, gaussians: dict, cams, targets, tile=(16, 16)):
    """The gradients of L = 1/2 sum_views ||C_v - target_v||^2 w.r.t. every Gaussian
    parameter, summed over the given views: one batched step through the library
    (projection, binning, forward, dL/dC = C - target, backward, projection backward)."""
    from . import raster
    V = len(cams)
    N = gaussians["means3D"].shape[0]
    if V == 0:
        return {k: torch.zeros_like(gaussians[k]) for k in GRAD_KEYS}
    pre = raster.preprocess_batched(plan, gaussians["means3D"], gaussians["log_scales"], gaussians["quats"],
                                    gaussians["opacities"], cams, tile)
    pl, rg, K = raster.bin_and_sort_batched(plan, pre["means2D"], pre["radii"], pre["depths"], cams, tile,
                                            conic_opacity=pre["conic_opacity"])
    outs = raster.render_forward_batched(plan, pre["means2D"], pre["conic_opacity"], gaussians["colors"],
                                         pre["depths"], pl, K, rg, cams, tile, mode="pixel")
    gin = [dict(color=o["color"] - t) for o, t in zip(outs, targets)]
    gr = raster.render_backward_batched(plan, pre["means2D"], pre["conic_opacity"], gaussians["colors"],
                                        pre["depths"], pl, K, rg, cams, outs, gin, tile, mode="pixel")
    gp = raster.preprocess_backward_batched(plan, gaussians["means3D"], gaussians["log_scales"], gaussians["quats"],
                                            cams, pre["radii"], gr["means2D"], gr["conic"])
    return dict(means3D=gp["means3D"], log_scales=gp["log_scales"], quats=gp["quats"],
                opacities=gr["opacity"].reshape(V, N).sum(0), colors=gr["colors"])


def sharded_gaussian_grads(plan, gaussians: dict, cams, targets, rank: int, world: int, group=None, loads=None,
                           tile=(16, 16)):
    """A rank's share of a multi-view training step: renders the views
    ``partition_views(cams, world, loads)[rank]`` and all-reduces the per-Gaussian gradients,
    so every rank ends with the gradients summed over all views."""
    mine = partition_views(cams, world, loads)[rank]
    g = local_gaussian_grads(plan, gaussians, [cams[v] for v in mine], [targets[v] for v in mine], tile)
    if world > 1:
        allreduce_gaussian_grads(g, group)
    return g, mine
