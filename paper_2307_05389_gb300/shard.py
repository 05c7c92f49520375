"""Bin-range sharding of one series over several ranks (one GPU each).

MinMax and M4 select points bin by bin, and each bin's selections depend on
that bin alone (Section 2.2 runs bins on separate threads).  So one series'
bins can be split across ranks: rank r of N owns the consecutive bins
``[floor(r*nb/N), floor((r+1)*nb/N))`` of the whole-series bin layout, runs the
bin-range entry point (``tsds_minmax_bins`` / ``tsds_m4_bins``) on them, which
reads only the part of y those bins cover, and the whole output is the
concatenation of the ranks' index lists in rank order.  The only exchange is
that final gather of variable-length index lists (``gather_indices``: an
all-gather of the counts, then of the lists padded to the longest).

Batched and served work shards by series instead (independent replicas); the
LTTB chain is sequential and does not shard.

This module is host logic over ``torch.distributed`` (NCCL for device
tensors, gloo for host tensors); it does none of the method's arithmetic.
"""
from __future__ import annotations

PER_BIN = {"minmax": 2, "m4": 4}


def shard_bins(nb: int, rank: int, world: int) -> tuple[int, int]:
    """The bins [b0, b1) that `rank` of `world` owns: near-equal consecutive ranges in rank
    order covering [0, nb)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if nb < 0:
        raise ValueError("nb must be >= 0")
    return nb * rank // world, nb * (rank + 1) // world


def gather_indices(local, group=None):
    """Concatenation in rank order of every rank's 1-D int64 tensor `local` (any lengths).

    Collective: every rank of `group` calls it.  The tensors stay on their device (CPU
    tensors with gloo, CUDA tensors with NCCL)."""
    import torch
    import torch.distributed as dist
    if local.dim() != 1 or local.dtype != torch.int64:
        raise ValueError("gather_indices takes a 1-D int64 tensor")
    world = dist.get_world_size(group)
    count = torch.tensor([local.numel()], dtype=torch.int64, device=local.device)
    counts = [torch.empty_like(count) for _ in range(world)]
    dist.all_gather(counts, count, group=group)
    sizes = [int(c.item()) for c in counts]
    width = max(max(sizes), 1)
    padded = torch.full((width,), -1, dtype=torch.int64, device=local.device)
    padded[:local.numel()] = local
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([p[:k] for p, k in zip(parts, sizes)])


def downsample_sharded(algo, y, n_out, x=None, nan="propagate", group=None):
    """MinMax or M4 of the whole series `y` (optional x) with the bins split over the ranks of
    `group`; every rank returns the whole output.  Each rank's y (and x) must be the whole
    series, resident on that rank's GPU (its kernels read only its bins' part)."""
    import torch.distributed as dist

    from . import binding
    if algo not in PER_BIN:
        raise ValueError(f"bin-range sharding covers MinMax and M4, not {algo!r}")
    n = y.shape[0]
    if n_out >= n:
        # every index: rank 0 contributes them all
        local = binding.downsample(algo, y, n_out, x=x, nan=nan)
        if dist.get_rank(group) != 0:
            local = local[:0]
        return gather_indices(local, group)
    nb = n_out // PER_BIN[algo]
    b0, b1 = shard_bins(nb, dist.get_rank(group), dist.get_world_size(group))
    local = binding.downsample_bins(algo, y, n_out, b0, b1, x=x, nan=nan)
    return gather_indices(local, group)
