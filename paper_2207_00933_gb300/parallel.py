"""Multi-GPU arrangement of the reconstruction (host side only).

The path partitions without any data-path exchange: every rank owns its own
circuits or its own slice of the output bins (a zoom prefix per rank), runs
the whole hot path on its GPU, and the ranks meet only to merge their
selected bins and to agree on timings.  These helpers are the host-side
pieces of that arrangement; they use torch.distributed (NCCL on GPUs, gloo
on CPU) and never touch the reconstruction's arithmetic.
"""
from __future__ import annotations

import numpy as np


def shard_prefix(rank: int, world: int) -> list[int]:
    """Bits of the zoom prefix that give rank `rank` its share of the bins:
    with world = 2^p ranks, rank r fixes p extra qubits to the bits of r
    (least significant first).  Returns the p bit values."""
    if world & (world - 1):
        raise ValueError("world size must be a power of two to split bins by a zoom prefix")
    p = world.bit_length() - 1
    return [(rank >> j) & 1 for j in range(p)]


def merge_top_bins(bins: np.ndarray, probs: np.ndarray, k: int, group=None):
    """Merge every rank's selected (bin, probability) pairs into the global
    k largest, ordered by probability descending then bin ascending (the
    order sqc_top_bins uses).  bins: global bin ids (int64), probs: float64.
    Returns the same result on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([len(bins)], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    cap = int(max(s.item() for s in sizes))
    b = torch.full((cap,), -1, dtype=torch.int64)
    v = torch.full((cap,), -np.inf, dtype=torch.float64)
    b[: len(bins)] = torch.as_tensor(np.asarray(bins, dtype=np.int64))
    v[: len(probs)] = torch.as_tensor(np.asarray(probs, dtype=np.float64))
    gb = [torch.empty_like(b) for _ in range(world)]
    gv = [torch.empty_like(v) for _ in range(world)]
    dist.all_gather(gb, b, group=group)
    dist.all_gather(gv, v, group=group)
    allb = torch.cat(gb).numpy()
    allv = torch.cat(gv).numpy()
    keep = allb >= 0
    allb, allv = allb[keep], allv[keep]
    order = np.lexsort((allb, -allv))[:k]
    return allb[order], allv[order]


def max_over_ranks(value: float, group=None) -> float:
    """The largest of every rank's value (timings: the slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
