"""Host-side logic for running the method on several GPUs (one process each).

The paper's two-GPU scheme (Sec. 3.1, last paragraph; Sec. 3.2, Fig. 2 and the
two-GPU stage list) generalises to P ranks as follows, and these helpers hold
its bookkeeping:

* HMF: particles are split into contiguous shards; each stage every rank sums
  cos and sin over its shard and the P partial sums are combined
  (`allreduce_sums`, in rank order, so every rank gets the same bits).
* Ring / 2D: i-rows are split into shards and every rank needs all positions;
  each stage the updated shards are gathered (`allgather_shards`) before the
  force pass over (own rows) x (all columns).
* Ensembles: independent systems are assigned to ranks by longest-processing-
  time first on N^2 (`lpt_assign`); no exchange at all.

They run on any torch.distributed backend (gloo on CPU in the tests).
"""
from __future__ import annotations

import numpy as np


def shard_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of n items owned by `rank` (sizes differ by at most 1)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def lpt_assign(costs, world: int) -> np.ndarray:
    """Rank of each item: longest-processing-time first onto the least-loaded rank
    (ties to the lowest rank), deterministic."""
    costs = np.asarray(costs, dtype=np.float64)
    order = np.argsort(-costs, kind="stable")
    load = np.zeros(world)
    owner = np.empty(costs.size, dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += costs[i]
    return owner


def allreduce_sums(local, group=None) -> np.ndarray:
    """Sum of every rank's FP64 vector, added in rank order on every rank."""
    import torch
    import torch.distributed as dist

    t = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64))
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out.numpy()


def allgather_shards(local, n: int, group=None) -> np.ndarray:
    """Concatenate each rank's shard (rank r owns shard_range(n, r, P)) into the full array."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    sizes = [shard_range(n, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    t = torch.zeros(width, dtype=torch.float64)
    loc = torch.as_tensor(np.ascontiguousarray(local, dtype=np.float64))
    t[: loc.numel()] = loc
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    return np.concatenate([parts[r][: hi - lo].numpy() for r, (lo, hi) in enumerate(sizes)])


def max_over_ranks(x: float, group=None) -> float:
    """The largest value of x over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
