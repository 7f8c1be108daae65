"""Checkpoint and resume on the GPU: a run stopped after two steps, saved and
restored into a new handle, repeats the uninterrupted run bit for bit (the
step starts from the committed fields alone: frozen data, coarse iterates and
error levels are all rebuilt), in FP64 and in mixed precision with the
coupled smoother."""
import numpy as np
import pytest

from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


@pytest.mark.parametrize("precision,coupled", [(0, 0), (1, 1)])
def test_resume_repeats_the_run(qn, tmp_path, precision, coupled):
    P = W.small_case(32, 48, False)
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=precision, coupled=coupled)
    a.set_fields(P.fields())
    for _ in range(2):
        a.step(P.dt)
    path = str(tmp_path / "ck.npz")
    a.save_checkpoint(path, t=2 * P.dt, n=2)
    b, t, n = qn.Solver.from_checkpoint(path)
    assert (t, n) == (2 * P.dt, 2) and b.options() == a.options()
    for _ in range(2):
        na, _ = a.step(P.dt)
        nb, _ = b.step(P.dt)
        assert na == nb
    fa, fb = a.get_fields(), b.get_fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_run_driver_log_and_resume(qn, tmp_path):
    """run.simulate on the GPU: the log shows mass conserved and the energy not
    increasing step by step; a run resumed from its checkpoint ends where the
    uninterrupted one does."""
    import json

    from paper_1703_06606_gb300 import run
    P = W.small_case(32, 32, True)
    a = qn.Solver(**P.create_kwargs(), tol=P.tol)
    a.set_fields(P.fields())
    ck, lg = str(tmp_path / "run.npz"), tmp_path / "run.jsonl"
    with open(lg, "w") as log:
        t, n = run.simulate(a, P.dt, 3, log=log, checkpoint=ck)
    recs = [json.loads(x) for x in lg.read_text().splitlines()]
    assert [r["step"] for r in recs] == [1, 2, 3] and all(r["status"] == 0 for r in recs)
    m0 = recs[0]["mass_rho"]
    assert all(abs(r["mass_rho"] - m0) <= 1e-12 * abs(m0) for r in recs)
    assert all(b["energy"] <= a_["energy"] for a_, b in zip(recs, recs[1:]))
    b, tb, nb = qn.Solver.from_checkpoint(ck)
    assert nb == 3 and tb == pytest.approx(3 * P.dt)
    run.simulate(a, P.dt, 2, t, n)
    run.simulate(b, P.dt, 2, tb, nb)
    fa, fb = a.get_fields(), b.get_fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
