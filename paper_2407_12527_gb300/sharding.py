"""Sample sharding of a ROM run over processes (one GPU each).

ROM samples are independent (Sec. 3.3 of the paper: the runs can be done in
parallel and averaged), so a run of n samples splits into contiguous sample
ranges, one per rank, each solved by its own context with
``rom_set_ordinates_seed_offset`` (global sample indices, so the draws are the
same as in one process).  The only exchange is at the end: the sums of phi
(``rom_get_partial_sum``) and the sample counts are added over the ranks.
"""
from __future__ import annotations

import numpy as np


def sample_range(rank: int, world: int, n_total: int):
    """(first, count) of the contiguous block of samples of `rank` (0 <= rank < world)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    base, extra = divmod(n_total, world)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def allreduce_average(partial_sum: np.ndarray, count: int, group=None) -> np.ndarray:
    """Global sample average from each rank's FP64 sum of phi and its sample count
    (torch.distributed all-reduce; any backend, CPU tensors)."""
    import torch
    import torch.distributed as dist

    buf = torch.from_numpy(np.ascontiguousarray(partial_sum, dtype=np.float64).ravel().copy())
    cnt = torch.tensor([float(count)], dtype=torch.float64)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(cnt, op=dist.ReduceOp.SUM, group=group)
    if cnt.item() <= 0:
        raise ValueError("no samples on any rank")
    return (buf / cnt.item()).numpy().reshape(np.shape(partial_sum))
