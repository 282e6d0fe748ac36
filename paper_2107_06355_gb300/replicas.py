"""Multi-process layout of independent lattices (one process per GPU).

The method's units of work are independent lattices, so N ranks share nothing on
the data path: each rank advances its own lattices, and the only collective is
the max-over-ranks of the timed duration (bench.py) or any user reduction.
"""
from __future__ import annotations


def shard_instances(sizes, world_size):
    """Assign instances (node counts in `sizes`) to ranks, largest first onto the
    least-loaded rank (longest-processing-time rule). Returns one sorted index
    list per rank; every instance appears exactly once."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    load = [0] * world_size
    shards = [[] for _ in range(world_size)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = min(range(world_size), key=lambda q: (load[q], q))
        shards[r].append(i)
        load[r] += sizes[i]
    return [sorted(s) for s in shards]


def max_over_ranks(value, device=None):
    """The maximum of a float over the ranks of the default process group (the value
    itself without one). Works with gloo (CPU tensors) and NCCL (CUDA tensors)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
