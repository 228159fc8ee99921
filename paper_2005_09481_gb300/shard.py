"""Channel sharding across GPUs (one process per GPU).

Frequency channels are independent after channelisation (Denman et al. 2020, section 2.3:
each GPU processes its own channels, with no GPU-to-GPU traffic), so N ranks split the
channels with no data-path collective.  The only cross-rank operations are host-side: the
timing reduction (slowest rank) and, optionally, gathering results for checking.
"""
from __future__ import annotations


def channels_for_rank(n_chan: int, rank: int, world: int) -> list[int]:
    """Contiguous block of channels owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n_chan < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_chan, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def owner_of(chan: int, n_chan: int, world: int) -> int:
    """Rank that owns channel `chan` under channels_for_rank."""
    base, extra = divmod(n_chan, world)
    cut = extra * (base + 1)
    return chan // (base + 1) if chan < cut else extra + (chan - cut) // max(base, 1)


def slowest(seconds: float, group=None) -> float:
    """Largest value over all ranks (the whole-job time of a weakly scaled step)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return seconds
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
