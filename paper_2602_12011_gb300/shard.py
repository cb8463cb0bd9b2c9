"""Data-parallel sharding of independent parameter samples across ranks (one process per GPU).

Samples are independent units of the likelihood, so ranks split a batch into contiguous shards,
evaluate them with no data-path collective, and only gather the per-sample results where a caller
needs them in one place (a sampler's driver). The timing helper takes the maximum over ranks.
Collectives go through torch.distributed (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations


def shard_bounds(n: int, rank: int, world: int):
    """[lo, hi) of rank's contiguous shard of n samples (sizes differ by at most one)."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside world %d" % (rank, world))
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def gather_results(local, n: int, world: int):
    """All-gather per-sample results of every rank's shard into the full [n, ...] tensor (rank order).
    local: this rank's torch tensor [hi - lo, ...]; shards are padded to equal size for the collective."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return local
    m = max(shard_bounds(n, r, world)[1] - shard_bounds(n, r, world)[0] for r in range(world))
    pad = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    bufs = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad)
    parts = []
    for r in range(world):
        lo, hi = shard_bounds(n, r, world)
        parts.append(bufs[r][: hi - lo])
    return torch.cat(parts, dim=0)


def max_over_ranks(seconds: float, device=None) -> float:
    """Maximum of a per-rank duration over all ranks (the job's wall time)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
