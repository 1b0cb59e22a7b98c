"""Multi-GPU host logic (one process per GPU, torch.distributed).

Targets are independent once the source cloud is known (each stencil reads
only its own neighbours), so the path shards without any data-path
collective: a rank takes a contiguous range of target ids and the whole
(small, replicated) source cloud.  The benchmark runs one independent
replica of the workload per rank (weak scaling); the only collective is the
max-reduction of the step time."""
from __future__ import annotations


def shard_targets(n_targets: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of the targets rank `rank` owns; ranges differ by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n_targets, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return units_per_rank * steps * world / (max_ms * 1e-3)
