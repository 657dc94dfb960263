"""Sharding of independent KKR solves over ranks (one process per GPU).

The solves of different atoms and energies are independent (each is its own M = I - t G),
so ranks share no data: every rank solves its own shard, and the only exchange is the
host-visible reduction of step times (max over ranks) used for whole-job throughput.
"""
from __future__ import annotations


def atom_range(rank: int, world: int, per_rank: int) -> range:
    """Global ids of the atoms of `rank` when every rank solves `per_rank` atoms (weak scaling)."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError("need 0 <= rank < world and per_rank >= 0")
    return range(rank * per_rank, (rank + 1) * per_rank)


def balance(work, world: int):
    """Split solves of unequal cost over `world` ranks: longest first, each to the currently
    least-loaded rank (ties to the lowest rank).  Returns one index list per rank, each in
    increasing order, covering every index exactly once."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += work[i]
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the value itself when
    no group is initialised).  `device` holds the reduction buffer: a CUDA device for NCCL,
    the CPU for gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
