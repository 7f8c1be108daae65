"""The continuous-batching server: requests admitted under a memory budget in
arrival order, each advanced one step at a time as soon as its previous step
finished, retired when done; each request's result is identical to running
it alone, and a small request's steps do not wait for a large one's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch, serve
    return qnsch, serve


def test_server_results_equal_alone_and_budget_respected(env):
    qnsch, serve = env
    reqs = serve.poisson_requests(6, rate=1000.0, seed=11, n_min=64, n_max=128, steps=3, dt=1e-4)
    srv = serve.Server(budget_bytes=1.0, max_slots=64)
    fps = [srv.footprint(r.problem) for r in reqs]
    srv.budget = 2 * max(fps)          # two of the largest at a time: the rest must queue
    out, fields = srv.run(reqs, keep_fields=True)
    assert srv.max_used_bytes <= srv.budget
    assert srv.max_resident < len(reqs)
    assert all(r.status == 0 and r.done_steps == 3 for r in out)
    assert max(r.admitted for r in out) > min(r.finished for r in out)  # someone waited for memory
    for r in out:
        P = r.problem
        s = qnsch.Solver(**P.create_kwargs(), tol=P.tol, precision=srv.precision,
                         coupled=srv.coupled)
        s.set_fields(P.fields())
        for _ in range(3):
            s.step(P.dt)
        alone = s.get_fields()
        for k in alone:
            assert np.array_equal(alone[k], fields[r.rid][k]), (r.rid, k)
    stats = serve.summarize(out, srv.wall, srv.max_resident)
    assert stats["failed"] == 0 and stats["value"] > 0


def test_small_request_steps_are_not_held_by_a_large_one(env):
    """A 768^2 drop and a 128^2 capillary wave served together: the small one
    finishes all its steps first, and its step latency is its own (well below
    the large one's), not the large one's step time."""
    qnsch, serve = env
    reqs = serve.poisson_requests(2, rate=1e6, seed=3, n_min=128, n_max=128, steps=6, dt=1e-4)
    big = reqs[0]
    big.problem.m1 = big.problem.m2 = 768
    big.problem.Cn = 2.5 / 768
    big.problem.Pe = 1.0 / big.problem.Cn
    big.steps = 3
    srv = serve.Server(budget_bytes=150e9)
    out, _ = srv.run(reqs)
    b, s = out
    assert b.status == 0 and s.status == 0
    assert s.done_steps == 6 and b.done_steps == 3
    assert s.finished < b.finished
    assert np.median(s.step_ms) < 0.5 * np.median(b.step_ms), (s.step_ms, b.step_ms)
    assert np.median(s.device_ms) < 0.5 * np.median(b.device_ms), (s.device_ms, b.device_ms)
