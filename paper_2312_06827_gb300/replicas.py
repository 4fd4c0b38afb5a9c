"""Host side of the multi-GPU form: independent replicas, one process per GPU.

The denoiser has no exchange step: streams and frames are independent units, so N GPUs run N
replicas of the workload, each on its own stream of frames, with no collective on the data
path.  The only collectives are the timing barrier and the maximum of the ranks' times; the
whole job's throughput is all ranks' units divided by that maximum (weak scaling: the work per
GPU is fixed).  These helpers hold that logic so that it can be exercised on CPU (gloo) as well
as under NCCL."""
from __future__ import annotations

import os


def rank_info():
    """(world, rank, local_rank) from the launcher's environment (1, 0, 0 when run alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_stream(rank: int) -> int:
    """Stream index of a rank's replica: rank 0 runs the canonical workload (stream 0), every
    other rank its own stream (a scene of the same kind and size with its own layout and noise,
    hence about the same cost)."""
    return int(rank)


def max_over_ranks(dist, value: float, device="cpu") -> float:
    """The maximum of a per-rank float over all ranks (the value itself without a process
    group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank_per_step: float, steps: int, t_max_s: float) -> float:
    """Units per second of the whole job: every rank processed units_per_rank_per_step in each of
    `steps` steps, and the job took as long as its slowest rank."""
    if t_max_s <= 0:
        raise ValueError("non-positive time")
    return world * units_per_rank_per_step * steps / t_max_s
