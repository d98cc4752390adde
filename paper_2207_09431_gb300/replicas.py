"""Running independent lattices on several GPUs (one process per GPU).

The step has no exchange between lattices, so several GPUs run replicas or
deal out the cases of an ensemble: rank r takes cases r, r + N, r + 2N, ...
The only collectives are on the host side of the measurement: the slowest
rank's time (the job's time) and the gathering of per-case results.  They go
through torch.distributed with whatever backend the process group uses (NCCL
on GPUs; gloo in the CPU tests).
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """The items rank `rank` of `world` handles: every world-th, from rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(items)[rank::world]


def unshard(parts):
    """Inverse of shard: per-rank lists (in rank order) back to the original order."""
    out = []
    n = sum(len(p) for p in parts)
    for i in range(n):
        out.append(parts[i % len(parts)][i // len(parts)])
    return out


def job_time_ms(ms: float, dist=None) -> float:
    """The job's time: the maximum over ranks (a plain value without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64)
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local, dist=None):
    """Per-case results of all ranks, in the original case order."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return list(local)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, list(local))
    return unshard(parts)
