"""Multi-GPU bookkeeping of the bench: the solves are independent, so N GPUs
run N replicas with no data-path collective.  Only the timing is reduced (the
maximum over ranks) and the work of all ranks is summed."""
from __future__ import annotations


def shard(total: int, rank: int, world: int):
    """Contiguous share [start, start + count) of `total` independent solves for
    `rank`; the shares of all ranks cover every solve exactly once."""
    base, extra = divmod(total, world)
    count = base + (1 if rank < extra else 0)
    start = rank * base + min(rank, extra)
    return start, count


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process
    group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_mlups(node_updates_all_ranks: float, seconds_max: float) -> float:
    """Whole-job throughput: node updates of all ranks over the slowest rank's
    time, in millions per second."""
    return node_updates_all_ranks / seconds_max / 1e6
