"""Host-side aggregation for N independent replicas (one process per GPU).

A single instance does not shard: every colour sweep of every level would need
a halo exchange.  bench.py therefore runs one replica of the workload per GPU
with no collective on the data path, and only the timing is combined: the
whole-job rate is the units all ranks processed over the slowest rank's time
(weak scaling: the work per GPU is fixed as N grows).
"""
from __future__ import annotations


def slowest(seconds, device="cpu"):
    """The largest of the ranks' `seconds` (all_reduce MAX over the default
    process group: NCCL with a CUDA device, gloo with the CPU); the value
    itself without an initialised group of more than one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds, world, device="cpu"):
    """(units of all ranks) / (slowest rank's seconds), and that time."""
    t = slowest(seconds, device)
    return world * units_per_rank / t, t
