"""Population sharding across ranks (one process per GPU).

Robots are independent (Section II-C: each robot's springs and masses only interact within the
robot), so a multi-GPU run splits one population into contiguous shards, one per rank.  The
generation's one exchange step is the fitness: each rank simulates its shard, an all-gather of
8 bytes per robot gives every rank the whole population's fitness, and every rank then runs the
same selection, crossover and mutation on the same (replicated) genome matrix.  The counter-based
generator and the deterministic kernels make the replicas bitwise equal, so no genome is sent.
Timing: a barrier around the timed region and the reduction of the timing; the whole-job
throughput is the units all ranks processed divided by the slowest rank's time (weak scaling:
the per-rank shard is fixed as the rank count grows)."""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the torchrun environment (1 process when unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def shard_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's population shard: distinct per rank, equal to base_seed on rank 0."""
    return int(base_seed) + 1000 * int(rank)


def shard_range(total: int, world: int, rank: int):
    """(first, count) of a contiguous split of `total` units over `world` ranks (the first
    total % world ranks take one extra)."""
    base, extra = divmod(int(total), int(world))
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)


def _reduce(x: float, op, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM, device)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(units_this_rank: float, seconds_this_rank: float, device=None):
    """Whole-job throughput (sum of units over ranks / max of times) and its parts."""
    units = sum_over_ranks(units_this_rank, device)
    secs = max_over_ranks(seconds_this_rank, device)
    return units / secs if secs > 0 else 0.0, units, secs


def gather_population_fitness(fit_local, world: int):
    """The whole population's fitness from every rank's shard (float64 tensors on the rank's
    device, or CPU tensors under gloo), concatenated in rank order: the all-gather that is the
    generation's exchange step.  Shards may differ in length by one (shard_range); they are padded
    to the longest for the collective and trimmed after."""
    import torch
    import torch.distributed as dist
    if world == 1 or not (dist.is_available() and dist.is_initialized()):
        return fit_local
    n = torch.tensor([fit_local.numel()], dtype=torch.int64, device=fit_local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(x.item()) for x in sizes]
    width = max(sizes)
    pad = torch.zeros(width, dtype=fit_local.dtype, device=fit_local.device)
    pad[:fit_local.numel()] = fit_local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:k] for p, k in zip(parts, sizes)])
