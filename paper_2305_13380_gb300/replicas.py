"""Timing of independent replicas across ranks.

Every workload here is a set of independent simulations, so a run on N GPUs
is N replicas with no data-path collective: each rank advances its own copy,
and only the clock is shared.  A barrier lines the ranks up on both sides of
the timed region and the slowest rank's device time stands for the job, so
the aggregate throughput is (units of all ranks) / max time.

The helpers work under any initialised process group (NCCL on GPUs, gloo on
CPU) and reduce to plain values when there is none or it has one rank."""
from __future__ import annotations

import torch
import torch.distributed as dist


def active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def world_size() -> int:
    return dist.get_world_size() if active() else 1


def barrier() -> None:
    if active():
        dist.barrier()


def _device() -> torch.device:
    # NCCL reduces device tensors only; gloo reduces host tensors
    if active() and dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(value: float) -> float:
    """The largest `value` of all ranks (every rank gets it)."""
    if not active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float) -> float:
    """The sum of `value` over all ranks (every rank gets it)."""
    if not active():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_local: float, ms_local: float) -> tuple[float, float]:
    """(units of all ranks per second over the slowest rank's time, that
    time in ms)."""
    ms = max_over_ranks(ms_local)
    units = sum_over_ranks(units_local)
    return units / (ms / 1e3), ms
