"""The serving loop's host logic on CPU, with a stand-in backend in place of
the qnsch binding: admission in arrival order under the memory budget and the
slot limit, continuous batching at step granularity (every resident request's
next step is queued as soon as its own previous step is seen finished, so
requests join while others are resident, leave when done, and a small request
never waits for a large one's steps), a failing request leaving without
disturbing the others, and the refusal of a request larger than the budget."""
import threading

import pytest

from paper_1703_06606_gb300 import serve
from paper_1703_06606_gb300 import workloads as W


class FakeBackend:
    """Solver / footprint with the binding's signatures.  A solver's footprint
    is m1 * m2 bytes; a launched step finishes after `polls(m1, m2)` polls
    (larger grids take longer).  The backend tracks the bytes and solvers
    alive, the order of step launches and which solvers had a step in flight
    at each launch."""

    def __init__(self, fail_names=(), polls=lambda m1, m2: 1):
        self.fail_names = set(fail_names)
        self.polls = polls
        self.live_bytes = self.max_live_bytes = 0
        self.live = self.max_live = 0
        self.created = []
        self.launches = []      # (name, names of the other solvers with a step in flight)
        self.lock = threading.Lock()

    def footprint(self, m1, m2, periodic_x=False, levels=0, precision=0, Lx=1.0):
        return m1 * m2

    def Solver(self, m1, m2, **kw):
        s = FakeSolver(self, m1, m2)
        s.kw = kw
        return s


class FakeSolver:
    def __init__(self, be, m1, m2):
        self.be, self.fp, self.steps, self.name = be, m1 * m2, 0, None
        self.need = be.polls(m1, m2)
        self.left = None  # polls until the launched step finishes
        with be.lock:
            be.live_bytes += self.fp
            be.live += 1
            be.max_live_bytes = max(be.max_live_bytes, be.live_bytes)
            be.max_live = max(be.max_live, be.live)
            be.created.append(self)

    def set_fields(self, f):
        self.name = f["name"]

    def get_fields(self):
        return {"steps": self.steps}

    def step_launch(self, dt):
        assert self.left is None, "a step is already in flight"
        with self.be.lock:
            busy = [s.name for s in self.be.created if s.left is not None]
            self.be.launches.append((self.name, busy))
        self.left = self.need

    def step_poll(self):
        assert self.left is not None, "no step launched"
        self.left -= 1
        if self.left > 0:
            return None
        self.left = None
        self.steps += 1
        code = -4 if self.name in self.be.fail_names else 0
        return 3, 1e-10, code, 0.5

    def close(self):
        with self.be.lock:
            self.be.live_bytes -= self.fp
            self.be.live -= 1


def _requests(sizes, steps):
    out = []
    for k, ((m1, m2), n) in enumerate(zip(sizes, steps)):
        P = W.small_case(m1, m2, False)
        P.name = "r%d" % k
        P.fields = (lambda name: (lambda: {"name": name}))(P.name)
        out.append(serve.Request(k, P, n, 0.0))
    return out


def test_admission_in_order_under_budget_and_slots():
    sizes = [(32, 32)] * 3 + [(64, 32)] * 2 + [(32, 32)] * 3
    reqs = _requests(sizes, [2, 5, 3, 1, 4, 2, 3, 1])
    be = FakeBackend()
    srv = serve.Server(budget_bytes=3 * 1024 + 512, max_slots=3, backend=be)
    reqs, fields = srv.run(reqs, keep_fields=True)
    assert [s.name for s in be.created] == ["r%d" % k for k in range(8)]  # FIFO
    assert be.max_live_bytes <= 3 * 1024 + 512 and be.max_live <= 3
    assert srv.max_used_bytes <= 3 * 1024 + 512
    assert be.live == 0 and be.live_bytes == 0  # every solver closed
    for r in reqs:
        assert r.status == 0 and r.done_steps == r.steps
        assert fields[r.rid] == {"steps": r.steps}
        assert r.admitted <= r.finished
    # continuous batching: some request's first step was launched while an
    # earlier request, admitted before it, still had steps in flight
    first = {}
    for k, (name, busy) in enumerate(be.launches):
        first.setdefault(name, (k, busy))
    assert any(busy and name != "r0" for name, (k, busy) in first.items())


def test_a_small_request_does_not_wait_for_a_large_ones_steps():
    """Steps at step granularity: a small request (one poll per step) does
    all its steps while a large request (40 polls per step) is still in its
    first one, and its recorded step latency is its own, not the large
    request's."""
    reqs = _requests([(128, 128), (16, 16)], [2, 6])
    be = FakeBackend(polls=lambda m1, m2: 40 if m1 * m2 > 1000 else 1)
    srv = serve.Server(budget_bytes=1e9, backend=be)
    reqs, _ = srv.run(reqs, poll_sleep_s=0.0)
    big, small = reqs
    assert big.status == 0 and small.status == 0
    assert small.done_steps == 6 and big.done_steps == 2
    # all of the small request's launches came while the large one had a step in flight
    small_launches = [busy for name, busy in be.launches if name == "r1"]
    assert len(small_launches) == 6 and all("r0" in busy for busy in small_launches[1:])
    assert small.finished < big.finished
    assert max(small.step_ms) < min(big.step_ms)


def test_a_failing_request_leaves_alone():
    reqs = _requests([(32, 32)] * 4, [3, 3, 3, 3])
    be = FakeBackend(fail_names={"r1"})
    srv = serve.Server(budget_bytes=1e9, backend=be)
    reqs, _ = srv.run(reqs)
    assert [r.status for r in reqs] == [0, -4, 0, 0]
    assert [r.done_steps for r in reqs] == [3, 1, 3, 3]
    assert [n for n, _ in be.launches].count("r1") == 1 and be.live == 0


def test_a_request_larger_than_the_budget_is_refused():
    reqs = _requests([(64, 64)], [1])
    srv = serve.Server(budget_bytes=1000, backend=FakeBackend())
    with pytest.raises(ValueError):
        srv.run(reqs)


def test_request_records():
    import json
    reqs = _requests([(32, 32)] * 3, [2, 1, 3])
    be = FakeBackend(fail_names={"r1"})
    reqs, _ = serve.Server(budget_bytes=1e9, backend=be).run(reqs)
    recs = [json.loads(json.dumps(serve.request_record(r))) for r in reqs]
    assert [(x["request"], x["status"], x["done_steps"]) for x in recs] == [
        (0, 0, 2), (1, -4, 1), (2, 0, 3)]
    for x in recs:
        assert len(x["step_ms"]) == len(x["vcycles"]) == len(x["device_ms"]) == x["done_steps"]
        assert x["arrival_s"] <= x["admitted_s"] <= x["finished_s"]
        assert x["latency_ms"] >= x["queue_wait_ms"] >= 0.0


def test_tuned_options_reach_the_matching_requests():
    """A tuned table's entry (autotune.key_of: device, grid, boundary,
    precision, smoother) applies its launch-shape options to the requests it
    matches, and to no other."""
    from paper_1703_06606_gb300 import autotune
    reqs = _requests([(32, 32), (64, 32), (32, 32)], [1, 1, 1])
    P = reqs[1].problem
    table = {autotune.key_of(P, 1, 1, 0, autotune.device_name()):
             {"options": {"fuse_cells32": 2048, "vanka_team_max32": 0}, "ms_per_step": 1.0}}
    be = FakeBackend()
    serve.Server(budget_bytes=1e9, backend=be, tuned_table=table).run(reqs)
    kws = {s.name: s.kw for s in be.created}
    assert kws["r1"]["fuse_cells32"] == 2048 and kws["r1"]["vanka_team_max32"] == 0
    assert "fuse_cells32" not in kws["r0"] and "fuse_cells32" not in kws["r2"]
    assert all(kw["precision"] == 1 and kw["coupled"] == 1 for kw in kws.values())


def test_base_options_reach_every_request_and_the_table_overrides_them():
    """base_options (for example THROUGHPUT_OPTIONS) go to every simulation the
    server creates; a matching tuned-table entry replaces the keys it names."""
    from paper_1703_06606_gb300 import autotune
    reqs = _requests([(32, 32), (64, 32)], [1, 1])
    P = reqs[1].problem
    table = {autotune.key_of(P, 1, 1, 0, autotune.device_name()):
             {"options": {"fuse_cells32": 512}, "ms_per_step": 1.0}}
    be = FakeBackend()
    serve.Server(budget_bytes=1e9, backend=be, tuned_table=table,
                 base_options=serve.THROUGHPUT_OPTIONS).run(reqs)
    kws = {s.name: s.kw for s in be.created}
    for k, v in serve.THROUGHPUT_OPTIONS.items():
        assert kws["r0"][k] == v
    assert kws["r1"]["fuse_cells32"] == 512
    assert all(kws["r1"][k] == v for k, v in serve.THROUGHPUT_OPTIONS.items()
               if k != "fuse_cells32")


def test_throughput_options_are_library_options():
    """Every key of THROUGHPUT_OPTIONS is an option the header documents and
    the checkpoint keeps, so a served simulation can be saved and resumed with
    its options."""
    import os
    from paper_1703_06606_gb300 import checkpoint
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    header = open(os.path.join(root, "include", "qnsch.h")).read()
    for k in serve.THROUGHPUT_OPTIONS:
        assert '"%s"' % k in header, k
        assert k in checkpoint.OPTIONS, k
