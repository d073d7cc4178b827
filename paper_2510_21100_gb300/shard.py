"""Host-side logic of the multi-GPU form: one process per GPU, images sharded across ranks.

Images are independent problems, so the path shards with no collective on the data: each rank
enhances its own images.  `torch.distributed` is used only to line the ranks up (a barrier) and to
take the slowest rank's step time; the job's throughput is every rank's pixels over that time
(weak scaling: the work per rank is fixed as ranks are added).
"""
from __future__ import annotations


def rank_image_seeds(rank: int, n_local: int, config: int = 1) -> list[int]:
    """Seeds of this rank's synthetic images: distinct across ranks, the same on every run."""
    from paper_2510_21100_gb300 import synth
    return [synth.seed_for(config, rank * n_local + k) for k in range(n_local)]


def shard_range(n_items: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous slice [lo, hi) of n_items (a batch's images) that `rank` takes; the slices of
    all ranks cover every item exactly once and differ in length by at most one."""
    if world < 1 or not 0 <= rank < world or n_items < 0:
        raise ValueError("need 0 <= rank < world and n_items >= 0")
    return n_items * rank // world, n_items * (rank + 1) // world


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the slowest rank's step time); `value` itself alone."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank_step: float, ms_step_max: float) -> float:
    """Whole-job rate: all ranks' units of one step over the slowest rank's step time (per second)."""
    if ms_step_max <= 0:
        raise ValueError("step time must be positive")
    return world * units_per_rank_step / (ms_step_max / 1000.0)
