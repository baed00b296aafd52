"""Host-side logic for running the simulator as independent replicas.

The echo synthesis needs no exchange between GPUs: every ADC entry is an
independent sum over facets, and every scene of a dataset is independent.
A multi-GPU job is therefore a set of replicas, one process per GPU, each
simulating its own share of the scenes; the only communication is the
reduction of timings and counters for reporting (max over ranks of the
elapsed time, sum over ranks of the work).  These helpers work with any
``torch.distributed`` backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import List, Optional


def shard_range(n_items: int, rank: int, world: int) -> range:
    """Contiguous block of item indices owned by ``rank`` (sizes differ by at
    most one; every index owned exactly once)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    base, extra = divmod(int(n_items), world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def shard_weighted(weights: List[float], rank: int, world: int) -> List[int]:
    """Greedy longest-first assignment of items with uneven costs (e.g. the
    facet counts of dataset scenes); deterministic, returns the item indices
    of ``rank`` in ascending order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    order = sorted(range(len(weights)), key=lambda i: (-float(weights[i]), i))
    load = [0.0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += float(weights[i])
    return [i for i in range(len(weights)) if owner[i] == rank]


def _device_for(group) -> Optional[str]:
    import torch.distributed as dist
    return "cuda" if dist.get_backend(group) == "nccl" else "cpu"


def reduce_scalar(value: float, op: str = "max", group=None) -> float:
    """All-reduce one float over the ranks ("max" or "sum"); identity when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = _device_for(group)
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM, group=group)
    return float(t.item())


def job_throughput(local_work: float, local_seconds: float, group=None) -> dict:
    """Whole-job throughput of replicas: total work over the slowest rank's
    time (the job ends when its last replica does)."""
    total = reduce_scalar(local_work, "sum", group)
    slowest = reduce_scalar(local_seconds, "max", group)
    return {"work": total, "seconds": slowest,
            "per_second": total / slowest if slowest > 0 else float("nan")}
