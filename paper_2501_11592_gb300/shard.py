"""Data-parallel sharding of a signal batch across ranks.

Signals that share A are independent problems (Eq. 3: the columns of
Y = A S + xi), so N GPUs each solve a contiguous slice of the batch with a
replicated A; nothing is exchanged on the data path.  Only the optional
gather of the outputs to one rank uses a collective.  With the image priors
(Eq. 6 and 7) the columns of an image are fitted together, so an image's W
columns must stay on one rank: pass unit=W and the slices are whole images.
"""
from __future__ import annotations


def shard_range(batch: int, rank: int, world: int, unit: int = 1) -> tuple[int, int]:
    """[begin, end) of the signals owned by `rank`: whole units of `unit`
    consecutive signals (an image's columns), the ranks' unit counts
    differing by at most one."""
    if world < 1 or not 0 <= rank < world or batch < 0 or unit < 1 or batch % unit:
        raise ValueError("bad shard arguments")
    q, r = divmod(batch // unit, world)
    begin = rank * q + min(rank, r)
    return begin * unit, (begin + q + (1 if rank < r else 0)) * unit


def gather_rows(local, batch: int, world: int, group=None, unit: int = 1):
    """All-gather per-signal output rows (first dimension = local signals)
    into the full batch order on every rank (slices as shard_range)."""
    import torch
    import torch.distributed as dist
    sizes = [shard_range(batch, r, world, unit) for r in range(world)]
    width = max(e - b for b, e in sizes)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([parts[r][: e - b] for r, (b, e) in enumerate(sizes)], dim=0)
