"""Sharding independent instances over GPUs (one process per GPU).

Batched and served simulations are independent units: nothing is exchanged
between them, so a multi-GPU run places whole instances on GPUs and needs no
collective on the data path.  The placement is a longest-processing-time
bin-pack: instances in decreasing order of expected cost (finest cells x
expected V-cycles per step x steps) each go to the GPU with the least cost so
far among those whose device-memory budget (qnsch_footprint of the instances
already there) still holds them.  Every rank computes the same placement from
the same list, so no rank has to send it.  After the run the ranks' summaries
are combined on the host (gather over the process group: gloo on CPU, NCCL
between GPUs): the whole-job rate is the cell-steps of all ranks over the
slowest rank's wall time.
"""
from __future__ import annotations

import math

# expected V-cycles per step when none is known: the mixed-precision coupled
# path's mean over the batched drop workload
DEFAULT_CYCLES = 9.0


def expected_cost(P, steps=1, cycles=DEFAULT_CYCLES):
    """Expected work of `steps` time steps of problem P, in cell-V-cycles."""
    return float(P.m1) * float(P.m2) * float(cycles) * float(steps)


def lpt_partition(costs, footprints, n_gpus, budget_bytes):
    """Place item k (cost costs[k], device bytes footprints[k]) on one of
    n_gpus GPUs, each holding at most budget_bytes.  Items go in decreasing
    cost (ties: lower index first) to the GPU with the least cost so far
    (ties: lower GPU index) among those it fits on.  Returns one sorted list
    of item indices per GPU; raises ValueError if an item fits on no GPU."""
    if n_gpus < 1:
        raise ValueError("need at least one GPU")
    if len(costs) != len(footprints):
        raise ValueError("one cost and one footprint per item")
    load = [0.0] * n_gpus
    used = [0.0] * n_gpus
    parts = [[] for _ in range(n_gpus)]
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    for k in order:
        best = None
        for g in range(n_gpus):
            if used[g] + footprints[k] > budget_bytes:
                continue
            if best is None or load[g] < load[best]:
                best = g
        if best is None:
            raise ValueError("item %d (%d bytes) fits on no GPU under a budget of %d bytes"
                             % (k, footprints[k], budget_bytes))
        parts[best].append(k)
        load[best] += costs[k]
        used[best] += footprints[k]
    return [sorted(p) for p in parts]


def makespan(costs, parts):
    """The largest per-GPU cost of a placement."""
    return max((sum(costs[k] for k in p) for p in parts), default=0.0)


def lower_bound(costs, n_gpus):
    """No placement can do better than this: the largest single item, or an
    even split of the total."""
    if not costs:
        return 0.0
    return max(max(costs), math.fsum(costs) / n_gpus)


def shard_problems(problems, rank, world, budget_bytes, footprint, steps=1,
                   cycles=DEFAULT_CYCLES):
    """The indices of `problems` that rank `rank` of `world` runs (the same
    placement on every rank).  footprint(P) -> device bytes of P."""
    costs = [expected_cost(P, steps, cycles) for P in problems]
    fps = [footprint(P) for P in problems]
    return lpt_partition(costs, fps, world, budget_bytes)[rank]


def shard_requests(requests, rank, world, budget_bytes, footprint, cycles=DEFAULT_CYCLES):
    """The requests (serve.Request) rank `rank` of `world` serves.  The budget
    bounds what a GPU holds at once, not over the whole stream, so it only
    refuses requests that fit on no GPU at all; the placement balances the
    expected cost of each request's steps."""
    costs = [expected_cost(r.problem, r.steps, cycles) for r in requests]
    fps = [footprint(r.problem) for r in requests]
    for k, fp in enumerate(fps):
        if fp > budget_bytes:
            raise ValueError("request %d needs %d bytes, more than the budget" % (k, fp))
    parts = lpt_partition(costs, [0.0] * len(costs), world, budget_bytes)
    return [requests[k] for k in parts[rank]]


def combine(summaries):
    """Whole-job numbers from the ranks' summaries (dicts with cell_steps,
    wall_s, requests, failed and, optionally, per-step latencies): cell-steps
    of all ranks over the slowest rank's wall time."""
    cell_steps = sum(s["cell_steps"] for s in summaries)
    wall = max(s["wall_s"] for s in summaries)
    out = {"value": cell_steps / wall if wall > 0 else 0.0, "unit": "cell-updates/s",
           "cell_steps": cell_steps, "wall_s": wall, "ranks": len(summaries),
           "requests": sum(s.get("requests", 0) for s in summaries),
           "failed": sum(s.get("failed", 0) for s in summaries),
           "per_rank_value": [s["cell_steps"] / s["wall_s"] if s["wall_s"] > 0 else 0.0
                              for s in summaries]}
    return out


def gather_summaries(summary):
    """Every rank's summary on every rank (all_gather_object over the default
    process group); the summary itself without a group of more than one rank."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [summary]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, summary)
    return out
