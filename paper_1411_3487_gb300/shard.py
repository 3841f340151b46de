"""Host-side sharding of independent chains over ranks (one GPU per rank).

Chains do not interact (no hydrodynamics), so a multi-GPU run is a set of
replicas: rank r owns a contiguous, disjoint range of job ids and steps its
own batch with no collective in the step loop.  Because the thermal noise is
keyed by (seed, job id, step, bead), a chain's trajectory does not depend on
which rank runs it.  The only exchange is the merge of per-chain FP64
observable accumulators when they are read out, done here by gathering every
rank's block and summing in rank order, so the result is the same on every
rank and for every world size that partitions the same chains.
"""
from __future__ import annotations

import numpy as np


def job_range(rank: int, world: int, n_total: int, base: int = 0) -> range:
    """Job ids of ``rank``: contiguous blocks, sizes differing by at most one."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    q, r = divmod(n_total, world)
    lo = rank * q + min(rank, r)
    hi = lo + q + (1 if rank < r else 0)
    return range(base + lo, base + hi)


def gather_chains(local: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """All ranks' per-chain rows ``local[n_local, ...]`` in job order, on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    loc = np.ascontiguousarray(local, dtype=np.float64)
    sizes = [len(job_range(r, world, n_total)) for r in range(world)]
    if loc.shape[0] != sizes[rank]:
        raise ValueError(f"rank {rank} holds {loc.shape[0]} chains, expected {sizes[rank]}")
    width = int(np.prod(loc.shape[1:])) if loc.ndim > 1 else 1
    pad = max(sizes)
    buf = torch.zeros(pad * width, dtype=torch.float64)
    buf[: loc.size] = torch.from_numpy(loc.reshape(-1))
    outs = [torch.zeros(pad * width, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    rows = [o[: s * width].numpy().reshape((s,) + loc.shape[1:]) for o, s in zip(outs, sizes)]
    return np.concatenate(rows, axis=0)


def merge_sums(local: np.ndarray, n_total: int, group=None) -> np.ndarray:
    """Sum of per-chain accumulator rows over all chains of all ranks, in job
    order (fixed summation order, independent of the world size)."""
    allrows = gather_chains(local, n_total, group)
    out = np.zeros(allrows.shape[1:], dtype=np.float64)
    for row in allrows:
        out += row
    return out
