"""Host-side logic of running the sweep on several GPUs, one process per GPU.

Rails are independent (the zone field of a rail depends on that rail alone),
so a device is partitioned by rails: rank k advances the contiguous rows
[r0, r1) of shard_rails() as a device of r1 - r0 rails with rail_base = r0.
The rail index is Philox counter word 1 and the placement key, so the rank
reproduces exactly those rows of the whole device, with no exchange on the
data path.  Whole device instances can be dealt out too (shard_instances:
instance i to rank i % world; the instance is counter word 3).  The only
collectives are the readout (the int64 sums of the ranks' current and
zone-count traces, when one device-wide trace is wanted) and the timing (the
maximum over ranks, which the whole-job throughput divides by).  Works with
any torch.distributed backend: gloo with CPU tensors, NCCL with CUDA tensors.
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np


def rank_info():
    """(rank, local_rank, world) from the launcher's environment (1 process if unset)."""
    import os
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def shard_rails(n_rails: int, rank: int, world: int):
    """(r0, r1): the contiguous rails of a device this rank advances.  The
    first n_rails % world ranks take one rail more than the others."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, m = divmod(int(n_rails), world)
    r0 = rank * q + min(rank, m)
    return r0, r0 + q + (1 if rank < m else 0)


def shard_instances(n_instances: int, rank: int, world: int) -> List[int]:
    """The instances this rank advances: every world-th, starting at rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return list(range(rank, n_instances, world))


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def sum_traces(J: np.ndarray, Zc: np.ndarray, device: Optional[str] = None):
    """Sum this rank's int64 traces over all ranks (returns numpy arrays);
    without an initialised process group the input is returned."""
    dist = _dist()
    if dist is None:
        return J, Zc
    import torch
    tJ = torch.from_numpy(np.ascontiguousarray(J, dtype=np.int64))
    tZ = torch.from_numpy(np.ascontiguousarray(Zc, dtype=np.int64))
    if device:
        tJ, tZ = tJ.to(device), tZ.to(device)
    dist.all_reduce(tJ, op=dist.ReduceOp.SUM)
    dist.all_reduce(tZ, op=dist.ReduceOp.SUM)
    return tJ.cpu().numpy(), tZ.cpu().numpy()


def max_over_ranks(x: float, device: Optional[str] = None) -> float:
    """The maximum of a per-rank scalar (a timed duration) over all ranks."""
    dist = _dist()
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(device: Optional[str] = None):
    dist = _dist()
    if dist is not None:
        dist.barrier()


def whole_job_rate(units_per_rank: Sequence[float], seconds_max: float) -> float:
    """Throughput of the whole job: all ranks' units over the slowest rank's time."""
    return float(sum(units_per_rank)) / seconds_max
