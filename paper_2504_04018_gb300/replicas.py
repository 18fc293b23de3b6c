"""Host logic of the multi-GPU run: independent replicas, no data-path exchange.

ESG answers each query independently (a query's pieces, search and merge touch
only the index and that query), and the index fits one GB300, so N GPUs run N
replicas of the whole path, each on its own batch. The only cross-rank traffic
is control: a barrier around the timed region and a MAX reduction of the
per-rank elapsed time, so that the reported throughput is the work of all
ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import torch


def max_over_ranks(value: float, device=None) -> float:
    """MAX of a per-rank float over the default process group (identity when
    no group is initialised). `device` is where the reduction tensor lives:
    a CUDA device under NCCL, the CPU under gloo."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_rate(units_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: units processed by all `world` replicas over
    `steps` steps, divided by the (max-over-ranks) elapsed milliseconds."""
    if total_ms <= 0:
        raise ValueError("elapsed time must be positive")
    return world * units_per_rank * steps / (total_ms / 1e3)
