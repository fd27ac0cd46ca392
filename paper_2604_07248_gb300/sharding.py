"""Multi-rank host logic of the split-step path (one process per GPU).

The path shards by independent units (realizations, beams, instances): Philox counters depend only
on the global realization index, so any partition reproduces the single-GPU screens exactly.  The
only exchange is the final merge of the FP64 per-pixel moment accumulators (S25, Welford), done
here with the pairwise update of Chan, Golub and LeVeque in fixed rank order, so the merged result
does not depend on timing.
"""
from __future__ import annotations

import numpy as np


def shard(total: int, rank: int, world: int) -> range:
    """Contiguous block of unit indices owned by `rank` (the first total % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def merge_moments(parts):
    """Merge (count, mean, m2) accumulators in the given order; m2 is the sum of squared deviations."""
    n, mean, m2 = 0, None, None
    for c, mu, s2 in parts:
        if c == 0:
            continue
        mu = np.asarray(mu, np.float64)
        s2 = np.asarray(s2, np.float64)
        if n == 0:
            n, mean, m2 = c, mu.copy(), s2.copy()
            continue
        tot = n + c
        d = mu - mean
        mean = mean + d * (c / tot)
        m2 = m2 + s2 + d * d * (n * c / tot)
        n = tot
    return n, mean, m2


def gather_merge(count: int, mean, m2, group=None):
    """All ranks send their accumulators to rank 0 (torch.distributed, CPU tensors, gloo or nccl
    with CPU staging); rank 0 returns the merged (count, mean, m2) in rank order, others None."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    mean_t = torch.as_tensor(np.asarray(mean, np.float64)).contiguous()
    m2_t = torch.as_tensor(np.asarray(m2, np.float64)).contiguous()
    cnt_t = torch.tensor([count], dtype=torch.int64)
    if rank == 0:
        cnts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        means = [torch.zeros_like(mean_t) for _ in range(world)]
        m2s = [torch.zeros_like(m2_t) for _ in range(world)]
    else:
        cnts = means = m2s = None
    dist.gather(cnt_t, cnts, dst=0, group=group)
    dist.gather(mean_t, means, dst=0, group=group)
    dist.gather(m2_t, m2s, dst=0, group=group)
    if rank != 0:
        return None
    return merge_moments([(int(c.item()), mu.numpy(), s2.numpy()) for c, mu, s2 in zip(cnts, means, m2s)])
