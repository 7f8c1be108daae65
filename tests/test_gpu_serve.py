"""The continuous-batching server: requests admitted under a memory budget in
arrival order, advanced together, retired when done; each request's result is
identical to running it alone."""
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
    srv.budget = 2 * max(fps)          # at most two resident at a time: the rest must queue
    out, fields = srv.run(reqs, keep_fields=True)
    assert srv.max_resident <= 2
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
