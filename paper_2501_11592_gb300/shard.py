"""Data-parallel sharding of a signal batch across ranks.

Signals that share A are independent problems (Eq. 3: the columns of
Y = A S + xi), so N GPUs each solve a contiguous slice of the batch with a
replicated A; nothing is exchanged on the data path.  Only the optional
gather of the outputs to one rank uses a collective.
"""
from __future__ import annotations


def shard_range(batch: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the signals owned by `rank`; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or batch < 0:
        raise ValueError("bad shard arguments")
    q, r = divmod(batch, world)
    begin = rank * q + min(rank, r)
    return begin, begin + q + (1 if rank < r else 0)


def gather_rows(local, batch: int, world: int, group=None):
    """All-gather per-signal output rows (first dimension = local signals)
    into the full batch order on every rank."""
    import torch
    import torch.distributed as dist
    sizes = [shard_range(batch, r, world) for r in range(world)]
    width = max(e - b for b, e in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: e - b] for r, (b, e) in enumerate(sizes)], dim=0)
