"""Host-side helpers for running the timestep on several GPUs of one node.

The single-mesh timestep does not shard: N ranks run N independent
replicas.  The batched workload shards by mesh: each rank advances its own
subset of the meshes, with no exchange during a step.  What ranks share is
only the bookkeeping below: which meshes a rank owns, and the slowest
rank's time.
"""
from __future__ import annotations


def lpt_shards(weights, world):
    """Assign items to ``world`` ranks by the longest-processing-time rule:
    items in decreasing weight, each to the rank with the smallest total so
    far (ties to the lowest rank).  Returns one sorted index list per rank.
    Every rank's total is within the largest weight of every other's."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += weights[i]
    return [sorted(s) for s in out]


def max_over_ranks(value, dist=None, device=None):
    """The largest ``value`` over all ranks of the default process group
    (the value itself without one).  ``device`` is where the reduction
    tensor lives (a CUDA device for NCCL, CPU for gloo)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
