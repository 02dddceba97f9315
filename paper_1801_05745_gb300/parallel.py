"""Multi-process layer of the lightcone library (torch.distributed).

The method shards in two ways (Sec. 2.4 builds a lightcone from
independently processed subvolumes whose maps are then combined; Sec. 3.2
averages over independent realisations):
  - subvolumes: each rank bins a contiguous shard of a box's particles and
    the int32 count maps are summed across ranks (one all-reduce);
  - realisations: each rank makes its own maps and keeps its own Welford
    state; the states are gathered in rank order and merged with the Chan
    update (ufc_welford_merge), which makes the result independent of how the
    realisations were split.
"""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int, align: int = 1) -> tuple[int, int]:
    """[start, stop) of rank's contiguous share of n particles; every start is
    a multiple of `align` (4 keeps a shard of 12-byte particles on 16-byte
    boundaries, which the binning's bulk copies need)."""
    units, rest = divmod(n, align)
    base, extra = divmod(units, world)
    start = (rank * base + min(rank, extra)) * align
    stop = start + (base + (1 if rank < extra else 0)) * align
    if rank == world - 1:
        stop += rest
    return start, stop


def allreduce_counts(counts, group=None):
    """Sums the partial count maps of all ranks in place (the combination of
    subvolume maps)."""
    import torch.distributed as dist
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def gather_states(state, group=None):
    """All ranks' Welford states, in rank order (every rank gets the list)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = [torch.empty_like(state) for _ in range(world)]
    dist.all_gather(out, state, group=group)
    return out


def merge_states(ctx, states, d: int):
    """Chan-merges gathered states in rank order; returns the merged state (a
    new tensor).  Device tensors merge on the device (ufc_welford_merge);
    host tensors, as a CPU transport gathers them, through
    ufc_welford_merge_host (ctx may then be None)."""
    merged = states[0].clone()
    if merged.is_cuda:
        for s in states[1:]:
            ctx.welford_merge(merged, s, d)
        return merged
    from . import api
    m = merged.numpy()
    for s in states[1:]:
        api.welford_merge_host(m, s.contiguous().numpy(), d)
    return merged
