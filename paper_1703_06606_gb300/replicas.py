"""Host-side aggregation for N independent replicas (one process per GPU).

A single instance does not shard: every colour sweep of every level would need
a halo exchange.  bench.py therefore runs one replica of the workload per GPU
with no collective on the data path, and only the timing is combined: the
whole-job rate is the units all ranks processed over the slowest rank's time
(weak scaling: the work per GPU is fixed as N grows).  Failures are detected
on the host: a rank whose phase failed says so in the same collective, and a
rank that died ends the others' next collective by the process-group timeout.
"""
from __future__ import annotations


# seconds a rank waits in a collective for the others before the collective
# fails (bench.py's process group): a replica that died makes the others'
# next collective end with an error instead of waiting for ever
PG_TIMEOUT_S = 900.0


class ReplicaFailed(RuntimeError):
    """Some rank's replica reported a failed phase; raised on every rank."""


def slowest(seconds, device="cpu", ok=True):
    """The largest of the ranks' `seconds` (all_reduce MAX over the default
    process group: NCCL with a CUDA device, gloo with the CPU); the value
    itself without an initialised group of more than one rank.  `ok` = False
    on any rank (its phase failed) raises ReplicaFailed on every rank, so that
    all of them stop at the same point and none reports a number."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        if not ok:
            raise ReplicaFailed("the replica's phase failed")
        return float(seconds)
    t = torch.tensor([float(seconds) if ok else 0.0, 0.0 if ok else 1.0], dtype=torch.float64,
                     device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if t[1].item() != 0.0:
        raise ReplicaFailed("a replica's phase failed on some rank")
    return float(t[0].item())


def whole_job_rate(units_per_rank, seconds, world, device="cpu", ok=True):
    """(units of all ranks) / (slowest rank's seconds), and that time."""
    t = slowest(seconds, device, ok)
    return world * units_per_rank / t, t
