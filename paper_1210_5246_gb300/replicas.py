"""Runs on several GPUs of one node: one process per GPU, no exchange on the data path.

The Godunov step of one grid has no dependence on another grid, and the batched Riemann
tubes are independent problems, so N ranks either advance their own replica of a grid
(weak scaling) or split a batch of tubes between them.  The only collectives are the
barrier that opens and closes a timed region and the max over ranks of its duration; a
sharded batch adds sums of per-rank counts.  Each call works with the ``gloo`` (CPU) and
the ``nccl`` (GPU) backend.
"""
from __future__ import annotations

import os

import numpy as np


def dist_env():
    """(rank, world_size, local_rank) from the launcher's environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> bool:
    """Join the process group when WORLD_SIZE > 1 (env:// rendezvous).  Returns whether a
    group is active."""
    import torch
    import torch.distributed as dist
    _, world, _ = dist_env()
    if world <= 1:
        return False
    if not dist.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return True


def active() -> bool:
    import torch.distributed as dist
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def _device():
    import torch
    import torch.distributed as dist
    return torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")


def barrier():
    if active():
        import torch.distributed as dist
        dist.barrier()


def _reduce(x: float, op) -> float:
    if not active():
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float) -> float:
    """The largest x over all ranks (the duration of a timed region that all ranks ran)."""
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.MAX)


def sum_over_ranks(x: float) -> float:
    import torch.distributed as dist
    return _reduce(x, dist.ReduceOp.SUM)


def whole_job_rate(units_per_rank: float, max_seconds: float) -> float:
    """Units all ranks processed / the slowest rank's time."""
    return sum_over_ranks(units_per_rank) / max_seconds


def tube_cost(length) -> np.ndarray:
    """Relative cost of a tube run to a fixed time: cells x steps, and the CFL step count
    grows with the cell count, so cost ~ length^2."""
    n = np.asarray(length, dtype=np.float64)
    return n * n


def shard_tubes(length, rank: int, world: int) -> np.ndarray:
    """Indices of the tubes rank ``rank`` of ``world`` runs: longest-processing-time-first
    assignment on ``tube_cost`` (ties broken by index, so every rank computes the same
    partition), returned in increasing order.  The shards are disjoint and cover all
    tubes."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    cost = tube_cost(length)
    order = np.lexsort((np.arange(len(cost)), -cost))
    load = np.zeros(world)
    owner = np.empty(len(cost), dtype=np.int64)
    for i in order:
        r = int(np.argmin(load))
        owner[i] = r
        load[r] += cost[i]
    return np.nonzero(owner == rank)[0]
