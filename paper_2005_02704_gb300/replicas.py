"""Replicas across GPUs.

Scans are independent, so N GPUs run N independent replicas: each rank owns a
disjoint shard of the scan stream (its own seeds / sensors) and there is no
collective on the data path.  The only communication is timing bookkeeping
for the benchmark: a barrier around the timed region and max / sum
reductions of per-rank numbers (one process per GPU, torch.distributed).
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed0(rank: int, scans_per_rank: int, base: int = 2000) -> int:
    """First scan seed of a rank's shard: ranks draw disjoint seed ranges."""
    return base + rank * scans_per_rank


def shard_scans(n_total: int, rank: int, world: int):
    """Contiguous split of n_total scan indices over the ranks."""
    per = n_total // world
    extra = n_total % world
    start = rank * per + min(rank, extra)
    return range(start, start + per + (1 if rank < extra else 0))


class Reducer:
    """Barrier and max / sum over ranks; identity when world == 1."""

    def __init__(self, world: int, device=None):
        self.world = world
        self.device = device

    def _all_reduce(self, x: float, op):
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return float(t.item())

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        if self.world == 1:
            return float(x)
        import torch.distributed as dist
        return self._all_reduce(x, dist.ReduceOp.MAX)

    def sum(self, x: float) -> float:
        if self.world == 1:
            return float(x)
        import torch.distributed as dist
        return self._all_reduce(x, dist.ReduceOp.SUM)
