"""The serving loop's host logic on CPU, with a stand-in backend in place of
the qnsch binding: admission in arrival order under the memory budget and the
slot limit, continuous batching (requests join while others are resident and
leave when done), a failing request leaving without disturbing the others,
and the refusal of a request larger than the budget."""
import pytest

from paper_1703_06606_gb300 import serve
from paper_1703_06606_gb300 import workloads as W


class FakeBackend:
    """Solver / Batch / footprint with the binding's signatures.  A solver's
    footprint is m1 * m2 bytes; the backend tracks the bytes and solvers alive
    and every batch it is asked to step."""

    def __init__(self, fail_names=()):
        self.fail_names = set(fail_names)
        self.live_bytes = self.max_live_bytes = 0
        self.live = self.max_live = 0
        self.created = []
        self.batches = []

    def footprint(self, m1, m2, periodic_x=False, levels=0, precision=0, Lx=1.0):
        return m1 * m2

    def Solver(self, m1, m2, **kw):
        s = FakeSolver(self, m1, m2)
        s.kw = kw
        return s

    def Batch(self, solvers):
        return FakeBatch(self, solvers)


class FakeSolver:
    def __init__(self, be, m1, m2):
        self.be, self.fp, self.steps, self.name = be, m1 * m2, 0, None
        be.live_bytes += self.fp
        be.live += 1
        be.max_live_bytes = max(be.max_live_bytes, be.live_bytes)
        be.max_live = max(be.max_live, be.live)
        be.created.append(self)

    def set_fields(self, f):
        self.name = f["name"]

    def get_fields(self):
        return {"steps": self.steps}

    def close(self):
        self.be.live_bytes -= self.fp
        self.be.live -= 1


class FakeBatch:
    def __init__(self, be, solvers):
        self.be, self.solvers = be, list(solvers)

    def step(self, dts):
        assert len(dts) == len(self.solvers)
        self.be.batches.append([s.name for s in self.solvers])
        st = []
        for s in self.solvers:
            s.steps += 1
            st.append(-4 if s.name in self.be.fail_names else 0)
        return st, [3] * len(self.solvers)

    def close(self):
        pass


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
    assert be.live == 0 and be.live_bytes == 0  # every solver closed
    for r in reqs:
        assert r.status == 0 and r.done_steps == r.steps
        assert fields[r.rid] == {"steps": r.steps}
        assert r.admitted <= r.finished
    # continuous batching: some batch holds a request that joined after another left
    joined = {n: i for i, b in reversed(list(enumerate(be.batches))) for n in b}
    assert any(joined[b[-1]] > 0 and joined[b[0]] < joined[b[-1]] for b in be.batches)


def test_a_failing_request_leaves_alone():
    reqs = _requests([(32, 32)] * 4, [3, 3, 3, 3])
    be = FakeBackend(fail_names={"r1"})
    srv = serve.Server(budget_bytes=1e9, backend=be)
    reqs, _ = srv.run(reqs)
    assert [r.status for r in reqs] == [0, -4, 0, 0]
    assert [r.done_steps for r in reqs] == [3, 1, 3, 3]
    assert be.batches[1] == ["r0", "r2", "r3"] and be.live == 0


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
        assert len(x["step_ms"]) == len(x["vcycles"]) == x["done_steps"]
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
