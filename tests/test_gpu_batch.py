"""Batches of independent instances (qnsch_batch_*): each instance's result is the
same alone and in a mix of uneven sizes and parameters, and a failing instance
does not disturb the others."""
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


def mix(with_drops):
    probs = [W.small_case(32, 32, True), W.small_case(64, 48, False, rho_ratio=10.0),
             W.small_case(48, 64, False), W.capillary_64()]
    if with_drops:  # high density ratios: these need the coupled smoother
        drops = W.batch_drops(n=6, seed=5)
        probs += [d for d in drops if d.m1 <= 128][:3]
    return probs


@pytest.mark.parametrize("precision,coupled", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_batch_results_equal_alone(qn, precision, coupled):
    probs = mix(with_drops=bool(coupled))
    alone, batch = [], []
    for P in probs:
        kw = dict(P.create_kwargs(), tol=P.tol, precision=precision, coupled=coupled)
        a = qn.Solver(**kw)
        b = qn.Solver(**kw)
        f = P.fields()
        a.set_fields(f)
        b.set_fields(f)
        alone.append(a)
        batch.append(b)
    B = qn.Batch(batch)
    dts = [P.dt for P in probs]
    for _ in range(2):
        st, cyc = B.step(dts)
        assert all(x == 0 for x in st), st
        for a, P, n in zip(alone, probs, cyc):
            na, _ = a.step(P.dt)
            assert na == n
    for a, b in zip(alone, batch):
        fa, fb = a.get_fields(), b.get_fields()
        for k in fa:
            assert np.array_equal(fa[k], fb[k]), k
        assert a.mass() == b.mass()


def test_batch_failure_is_isolated(qn):
    probs = mix(False)[:3]
    sol = [qn.Solver(**P.create_kwargs(), tol=P.tol) for P in probs]
    sol[1].set_option("maxcyc", 1)
    sol[1].set_option("tol", 1e-15)
    for sv, P in zip(sol, probs):
        sv.set_fields(P.fields())
    B = qn.Batch(sol)
    st, cyc = B.step([P.dt for P in probs])
    assert st[0] == 0 and st[2] == 0 and st[1] == -4
    assert cyc[1] == 1
    ref = qn.Solver(**probs[2].create_kwargs(), tol=probs[2].tol)
    ref.set_fields(probs[2].fields())
    ref.step(probs[2].dt)
    assert np.array_equal(ref.get_fields()["c"], sol[2].get_fields()["c"])


@pytest.mark.parametrize("max_inflight", [1, 2])
def test_batch_with_a_window_equals_alone(qn, max_inflight):
    """max_inflight: at most that many members step at once, the rest start as
    they finish; each member's result is still the one it has alone."""
    probs = mix(with_drops=False)
    alone, batch = [], []
    for P in probs:
        kw = dict(P.create_kwargs(), tol=P.tol, precision=1, coupled=1)
        a, b = qn.Solver(**kw), qn.Solver(**kw)
        a.set_fields(P.fields())
        b.set_fields(P.fields())
        alone.append(a)
        batch.append(b)
    B = qn.Batch(batch, max_inflight=max_inflight)
    st, cyc = B.step([P.dt for P in probs])
    assert all(x == 0 for x in st), st
    for a, b, P, n in zip(alone, batch, probs, cyc):
        na, _ = a.step(P.dt)
        assert na == n
        fa, fb = a.get_fields(), b.get_fields()
        assert all(np.array_equal(fa[k], fb[k]) for k in fa)
    t = B.step_times()
    assert t.shape == (len(probs),) and np.all(t > 0.0)
    with pytest.raises(qn.QnschError):
        B.set_option("max_inflight", -1)
    with pytest.raises(qn.QnschError):
        B.set_option("no_such_option", 1)
