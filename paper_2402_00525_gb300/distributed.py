"""Several GPUs on one scene: views shard over ranks, gradients meet in one all-reduce.

The views of a scene are independent in the forward pass (Sec. 3: every view runs its own
Preprocess, sort and Render), so ranks render disjoint view subsets with no exchange. A training
step on one scene differentiates the sum of the per-view losses, and the backward pass of each
rank accumulates (+=) the gradients of its own views into the scene's parameter-shaped buffers
(Sec. 3.5). The one exchange is therefore a sum of those buffers over the ranks, after every
rank's backward; each rank then holds the gradient of the whole step. Scenes rendered on
different ranks need no exchange at all.

torch.distributed is only the transport (NCCL between GPUs, gloo on CPU); the buffers are the
ones libstp's backward wrote.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Union

import torch

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def shard_views(cams: Sequence, rank: int, world: int) -> list:
    """Views of rank `rank` of `world`: rank r takes views r, r + world, ... (each view once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    return list(cams)[rank::world]


def allreduce_gradients(grads: Union[Dict[str, torch.Tensor], List[Dict[str, torch.Tensor]]],
                        group=None, average: bool = False) -> None:
    """Sum (or average) per-scene gradient buffers over the ranks of `group`, in place.

    grads is one dict of parameter-shaped tensors (one scene) or a list of such dicts (several
    scenes, each summed separately). All buffers that share a device and dtype travel in one
    flattened all-reduce, so a step costs one collective whatever the number of fields. Every
    rank must pass buffers of the same shapes in the same order."""
    import torch.distributed as dist
    scenes = [grads] if isinstance(grads, dict) else list(grads)
    tensors = [s[k] for s in scenes for k in FIELDS]
    if not tensors:
        return
    groups: Dict[tuple, List[torch.Tensor]] = {}
    for t in tensors:
        groups.setdefault((t.device, t.dtype), []).append(t)
    world = dist.get_world_size(group)
    for ts in groups.values():
        flat = torch.cat([t.reshape(-1) for t in ts])
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        if average:
            flat /= world
        off = 0
        for t in ts:
            n = t.numel()
            t.copy_(flat[off:off + n].view_as(t))
            off += n


def gradient_buffers(g: dict) -> tuple:
    """(flat, grads): one zeroed float32 buffer on the scene's device and, in `grads`, views of
    it shaped like the scene's parameters. A backward that accumulates into `grads` leaves the
    whole gradient in `flat`, which allreduce_buffer() sums with no copy."""
    sizes = [g[k].numel() for k in FIELDS]
    flat = torch.zeros(sum(sizes), dtype=torch.float32, device=g[FIELDS[0]].device)
    grads, off = {}, 0
    for k, n in zip(FIELDS, sizes):
        grads[k] = flat[off:off + n].view(g[k].shape)
        off += n
    return flat, grads


def allreduce_buffer(flat: torch.Tensor, group=None, average: bool = False) -> None:
    """Sum (or average) a flat gradient buffer from gradient_buffers() over the ranks, in place."""
    import torch.distributed as dist
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    if average:
        flat /= dist.get_world_size(group)
