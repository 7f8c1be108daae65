"""The N > 1 host logic of bench.py on CPU: two gloo ranks with different
times agree on the slowest one, and the whole-job rate counts every rank's
units over it."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    from paper_1703_06606_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.5][rank]
        rate, t = replicas.whole_job_rate(1000.0, seconds, world)
        out.put((rank, rate, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, rate, t in res:
        assert t == 2.5
        assert rate == pytest.approx(2 * 1000.0 / 2.5)


def test_single_process_is_its_own_slowest():
    from paper_1703_06606_gb300 import replicas
    rate, t = replicas.whole_job_rate(10.0, 0.5, 1)
    assert t == 0.5 and rate == 20.0


def _rank_fails(rank, world, port, out):
    import torch.distributed as dist
    from paper_1703_06606_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        replicas.slowest(1.0, ok=(rank == 0))
        out.put((rank, "returned"))
    except replicas.ReplicaFailed:
        out.put((rank, "ReplicaFailed"))
    finally:
        dist.destroy_process_group()


def test_a_failed_replica_stops_every_rank():
    """Rank 1's phase fails: both ranks raise ReplicaFailed at the same
    collective and neither reports a time."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_fails, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, "ReplicaFailed"), (1, "ReplicaFailed")]


def _rank_dies(rank, world, port, out):
    import datetime
    import time
    import torch.distributed as dist
    from paper_1703_06606_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)  # leaves between phases, without joining the next collective
    t0 = time.time()
    try:
        replicas.slowest(1.0)
        out.put((rank, "returned", time.time() - t0))
    except Exception as e:  # the backend's error type differs between versions
        out.put((rank, type(e).__name__, time.time() - t0))


def test_a_dead_rank_ends_the_next_collective():
    """A rank that exits between phases makes the other's next collective fail
    within the process-group timeout instead of waiting for ever."""
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_dies, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what, waited = out.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert rank == 0 and what != "returned" and waited < 60.0, (what, waited)
