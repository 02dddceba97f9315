"""Multi-process layer of the lightcone library (torch.distributed).

The method shards in two ways (Sec. 2.4 builds a lightcone from
independently processed subvolumes whose maps are then combined; Sec. 3.2
averages over independent realisations):
  - subvolumes: each rank bins a contiguous shard of a box's particles;
    kappa is linear in the counts, so the ranks' FP64 partial sums
    sum_b A_b n_bp (8 B per pixel) are all-reduced and every rank finishes
    the map, and the adjoint's per-shell sums are all-reduced (4 doubles per
    shell) instead of the count maps (4 B per shell and pixel); summing the
    int32 count maps is the alternative when the counts are wanted;
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


def _active() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized()


def allreduce_adjoint_sums(sums, nshell: int, group=None, device=None):
    """Combines the ranks' adjoint sums (layout of ufc_kappa_adjoint_sums):
    the first 4 nshell entries are each rank's share of the per-shell sums and
    are summed; the last 4 are power sums of the whole map, which every rank
    computed from the same summed partials, so they are not summed: an
    all-reduce of their maxima and negated minima checks that the ranks agree
    (to 1e-9 relative: GPUs with other SM counts sum in another order) and
    every rank takes the maxima, so that all ranks return the same array.
    `device` is where the collective runs (a CUDA device under NCCL).
    Returns a new host FP64 array."""
    import numpy as np
    import torch
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    if sums.shape != (4 * nshell + 4,):
        raise ValueError("adjoint sums need 4 nshell + 4 entries")
    if not _active():
        return sums.copy()
    import torch.distributed as dist
    t = torch.from_numpy(sums.copy())
    if device is not None:
        t = t.to(device)
    head = t[:4 * nshell].contiguous()
    tail = t[4 * nshell:]
    ext = torch.cat([tail, -tail])
    dist.all_reduce(head, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(ext, op=dist.ReduceOp.MAX, group=group)
    hi, lo = ext[:4].cpu().numpy(), -ext[4:].cpu().numpy()
    if np.any(np.abs(hi - lo) > 1e-9 * np.maximum(np.abs(hi), np.abs(lo))):
        raise RuntimeError("ranks disagree on the whole-map power sums: their summed partial "
                           "maps differ")
    return np.concatenate([head.cpu().numpy(), hi])


def subvolume_kappa(ctx, counts, A, C, pdf_lo, pdf_hi, nbins, dA=None, dC=None, w_var=0.0,
                    w_skew=0.0, g_kappa=None, kappa=None, partial=None, group=None):
    """The map of a lightcone whose subvolumes were binned by different ranks
    (Sec. 2.4), on every rank: the rank's FP64 partial sum of its own counts
    (ufc_kappa_partial), one all-reduce of the partials, then the map, its
    moments and PDF (ufc_kappa_stats_partial).  With dA and dC also the
    gradient of L = w_var var + w_skew skew + <g, kappa>: the same read of the
    counts gives the map and the rank's share of the adjoint sums
    (ufc_kappa_adjoint_sums), the per-shell sums are all-reduced and the
    chain rule runs on the host (ufc_kappa_grad_from_sums).
    Returns (kappa, moments, pdf) or (kappa, moments, pdf, grad, G, H)."""
    from . import api
    partial = ctx.kappa_partial(counts, A, out=partial)
    if _active():
        import torch.distributed as dist
        dist.all_reduce(partial, op=dist.ReduceOp.SUM, group=group)
    if dA is None:
        return ctx.kappa_stats_partial(partial, C, pdf_lo, pdf_hi, nbins, kappa=kappa)
    S, npix = counts.shape
    nside = int(round((npix / 12) ** 0.5))
    sums, kappa, mom, pdf = ctx.kappa_adjoint_sums(counts, partial, C, g_kappa, pdf_lo, pdf_hi,
                                                   nbins, kappa=kappa, want_map=True)
    sums = allreduce_adjoint_sums(sums, S, group, device=partial.device)
    grad, G, H = api.kappa_grad_from_sums(sums, S, nside, dA, dC, w_var, w_skew)
    return kappa, mom, pdf, grad, G, H
