"""Sharding independent instances over GPUs (paper_1703_06606_gb300/shard.py),
on CPU: the longest-processing-time placement puts every instance on exactly
one GPU, respects each GPU's memory budget, is deterministic, and stays within
Graham's bound of the optimum (checked against brute force on small cases);
the 64-drop batch splits evenly over 2, 4 and 8 GPUs; and two gloo ranks each
serve their share of a request stream (stand-in backend) and agree on the
combined whole-job numbers."""
import itertools
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1703_06606_gb300 import shard
from paper_1703_06606_gb300 import workloads as W


def _optimum(costs, n):
    best = float("inf")
    for assign in itertools.product(range(n), repeat=len(costs)):
        load = [0.0] * n
        for c, g in zip(costs, assign):
            load[g] += c
        best = min(best, max(load))
    return best


def test_every_item_placed_once_and_deterministic():
    costs = [5, 3, 8, 1, 9, 2, 7, 4, 6, 6]
    fps = [1] * len(costs)
    a = shard.lpt_partition(costs, fps, 3, 100)
    b = shard.lpt_partition(list(costs), list(fps), 3, 100)
    assert a == b
    assert sorted(k for p in a for k in p) == list(range(len(costs)))


@pytest.mark.parametrize("seed", range(6))
def test_within_grahams_bound_of_the_optimum(seed):
    import random
    rng = random.Random(seed)
    n = 2 + seed % 2
    costs = [rng.randint(1, 50) for _ in range(7)]
    parts = shard.lpt_partition(costs, [0] * len(costs), n, 1)
    opt = _optimum(costs, n)
    assert shard.makespan(costs, parts) <= (4.0 / 3.0 - 1.0 / (3 * n)) * opt + 1e-9
    assert opt >= shard.lower_bound(costs, n) - 1e-9


def test_budget_is_respected_and_forces_spreading():
    costs = [10, 9, 1, 1]
    fps = [6, 6, 1, 1]
    parts = shard.lpt_partition(costs, fps, 2, 8)
    for p in parts:
        assert sum(fps[k] for k in p) <= 8
    assert {0, 1} not in [set(p) for p in parts]
    with pytest.raises(ValueError):
        shard.lpt_partition([1, 1], [9, 1], 2, 8)
    with pytest.raises(ValueError):
        shard.lpt_partition([5, 5, 5], [6, 6, 6], 2, 8)  # the third fits nowhere


@pytest.mark.parametrize("world", [2, 4, 8])
def test_batch_workload_splits_evenly(world):
    probs = W.batch_drops(n=64)
    costs = [shard.expected_cost(P) for P in probs]
    fps = [P.m1 * P.m2 * 500.0 for P in probs]  # a stand-in footprint, ~500 B per cell
    parts = shard.lpt_partition(costs, fps, world, 150e9)
    assert sorted(k for p in parts for k in p) == list(range(64))
    assert shard.makespan(costs, parts) <= 1.1 * shard.lower_bound(costs, world)
    mine = [shard.shard_problems(probs, r, world, 150e9, lambda P: P.m1 * P.m2 * 500.0)
            for r in range(world)]
    assert mine == parts


def test_requests_split_disjointly():
    from paper_1703_06606_gb300 import serve
    reqs = serve.poisson_requests(40, rate=50.0, steps=5, n_min=128, n_max=1024)
    shares = [shard.shard_requests(reqs, r, 3, 150e9, lambda P: P.m1 * P.m2 * 500.0)
              for r in range(3)]
    ids = sorted(r.rid for s in shares for r in s)
    assert ids == list(range(40))
    costs = [sum(shard.expected_cost(r.problem, r.steps) for r in s) for s in shares]
    assert max(costs) <= 1.1 * sum(costs) / 3
    with pytest.raises(ValueError):
        shard.shard_requests(reqs, 0, 3, 10.0, lambda P: P.m1 * P.m2 * 500.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _serve_rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_1703_06606_gb300 import serve
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import test_serve_host as fake
        reqs = fake._requests([(32, 32), (64, 32), (16, 16), (32, 64), (16, 32)],
                              [3, 2, 5, 1, 4])
        mine = shard.shard_requests(reqs, rank, world, 1e9, lambda P: P.m1 * P.m2)
        be = fake.FakeBackend()
        srv = serve.Server(budget_bytes=1e9, backend=be)
        done, _ = srv.run(mine, poll_sleep_s=0.0)
        local = serve.summarize(done, srv.wall, srv.max_resident)
        allsum = shard.gather_summaries(local)
        out.put((rank, sorted(r.rid for r in done), shard.combine(allsum)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_serve_their_shares_and_agree():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    env_path = os.path.dirname(os.path.abspath(__file__))
    old = os.environ.get("PYTHONPATH", "")
    os.environ["PYTHONPATH"] = env_path + (os.pathsep + old if old else "")
    try:
        procs = [ctx.Process(target=_serve_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        res = sorted((out.get(timeout=120) for _ in procs), key=lambda x: x[0])
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    finally:
        os.environ["PYTHONPATH"] = old
    ids = sorted(res[0][1] + res[1][1])
    assert ids == [0, 1, 2, 3, 4] and not set(res[0][1]) & set(res[1][1])
    a, b = res[0][2], res[1][2]
    assert a == b
    cells = {0: 32 * 32 * 3, 1: 64 * 32 * 2, 2: 16 * 16 * 5, 3: 32 * 64 * 1, 4: 16 * 32 * 4}
    assert a["cell_steps"] == sum(cells.values())
    assert a["requests"] == 5 and a["failed"] == 0 and a["ranks"] == 2
