"""Failure detection and refusals, made on the host without any GPU fault:
step_time_limit ends a step with QNSCH_ETIMEOUT, diverge_cycles ends a
diverging step early with QNSCH_ENOTCONV, the device-memory budget refuses a
creation or a mixed-precision step with QNSCH_EBUDGET, out-of-range option
values and time steps give QNSCH_EINVAL, and allocation failures injected
through a caller's allocator give QNSCH_ENOMEM with every block returned.
Each failure leaves the committed state as it was and the handle usable."""
import ctypes
import gc

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


def _pair(qn, P, **opts):
    out = []
    for _ in range(2):
        s = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
        s.set_fields(P.fields())
        out.append(s)
    return out


def _same(a, b):
    fa, fb = a.get_fields(), b.get_fields()
    return all(np.array_equal(fa[k], fb[k]) for k in fa)


def test_step_time_limit(qn):
    """A limit far below one cycle's time stops the step before its first
    cycle; the state stays at level n and, with the limit lifted, the next
    step gives exactly what an untouched handle gives."""
    P = W.small_case()
    a, b = _pair(qn, P)
    f0 = a.get_fields()
    a.set_option("step_time_limit", 1e-9)
    with pytest.raises(qn.QnschError) as e:
        a.step(P.dt)
    assert e.value.code == -6
    f1 = a.get_fields()
    assert all(np.array_equal(f0[k], f1[k]) for k in f0)
    a.set_option("step_time_limit", 0.0)
    na, _ = a.step(P.dt)
    nb, _ = b.step(P.dt)
    assert na == nb and _same(a, b)


def test_step_time_limit_in_a_batch(qn):
    """In a batch only the instance with the limit times out; the others step
    as they do alone."""
    probs = [W.small_case(), W.small_case(48, 64, False), W.capillary_64()]
    batch, alone = [], []
    for P in probs:
        x, y = _pair(qn, P)
        batch.append(x)
        alone.append(y)
    batch[1].set_option("step_time_limit", 1e-9)
    f0 = batch[1].get_fields()
    st, _ = qn.Batch(batch).step([P.dt for P in probs])
    assert st == [0, -6, 0], st
    f1 = batch[1].get_fields()
    assert all(np.array_equal(f0[k], f1[k]) for k in f0)
    for i in (0, 2):
        alone[i].step(probs[i].dt)
        assert _same(batch[i], alone[i])


def test_diverge_cycles_stops_a_diverging_step(qn):
    """omega_vanka = 2.5 makes the smoother diverge (the residual grows by
    orders of magnitude every cycle).  With diverge_cycles = 2 the step ends
    after two cycles of growth with QNSCH_ENOTCONV instead of running to a
    non-finite residual; the state stays at level n."""
    P = W.small_case()
    s = qn.Solver(**P.create_kwargs(), tol=P.tol, omega_vanka=2.5, diverge_cycles=2, maxcyc=50)
    s.set_fields(P.fields())
    f0 = s.get_fields()
    n, r = ctypes.c_int(), ctypes.c_double()
    rc = qn.lib().qnsch_step(s._h, float(P.dt), ctypes.byref(n), ctypes.byref(r))
    assert rc == -4 and n.value == 2, (rc, n.value, r.value)
    f1 = s.get_fields()
    assert all(np.array_equal(f0[k], f1[k]) for k in f0)


def test_diverge_cycles_keeps_a_converging_step(qn):
    """The capillary wave's first step grows its residual over the first cycle
    and then converges; diverge_cycles = 2 leaves it, and its result, as it is."""
    P = W.capillary_64()
    a, b = _pair(qn, P)
    a.set_option("diverge_cycles", 2)
    for _ in range(2):
        na, _ = a.step(P.dt)
        nb, _ = b.step(P.dt)
        assert na == nb
    assert _same(a, b)


def test_budget_refuses_and_releases(qn):
    """Each handle reserves its footprint; a creation past the budget fails with
    QNSCH_EBUDGET, destroying a handle gives its bytes back, and a mixed step
    reserves its error levels' bytes (footprint at precision 1) or is refused."""
    P = W.small_case()
    fp0 = qn.footprint(P.m1, P.m2, P.periodic_x, P.levels, 0, P.Lx)
    fp1 = qn.footprint(P.m1, P.m2, P.periodic_x, P.levels, 1, P.Lx)
    # handles of earlier tests held by reference cycles are freed now, and no
    # automatic collection frees one while the counts are compared
    gc.collect()
    gc.disable()
    _, u0 = qn.budget()
    try:
        # room for one handle, not for a second one nor for its error levels
        assert fp0 < fp1 < 2 * fp0
        qn.set_budget(u0 + fp0 + (fp1 - fp0) // 2)
        a = qn.Solver(**P.create_kwargs(), tol=P.tol)
        assert qn.budget()[1] == u0 + fp0
        with pytest.raises(qn.QnschError) as e:
            qn.Solver(**P.create_kwargs(), tol=P.tol)
        assert e.value.code == -7
        assert qn.budget()[1] == u0 + fp0
        a.set_fields(P.fields())
        a.set_option("precision", 1)
        with pytest.raises(qn.QnschError) as e:
            a.step(P.dt)
        assert e.value.code == -7
        qn.set_budget(u0 + fp1)
        a.step(P.dt)
        assert qn.budget()[1] == u0 + fp1
        a.close()
        assert qn.budget()[1] == u0
        b = qn.Solver(**P.create_kwargs(), tol=P.tol)
        b.close()
    finally:
        qn.set_budget(0)
        gc.enable()


def test_option_values_out_of_range_are_refused(qn):
    """A refused value gives QNSCH_EINVAL and leaves the option as it was (a NaN
    tol would otherwise end every step before its first cycle)."""
    s = qn.Solver(16, 16)
    bad = [("tol", float("nan")), ("tol", -1.0), ("tol", float("inf")), ("nu1", -1),
           ("nu2", 1.5), ("nu_coarse", 1001), ("maxcyc", -2), ("omega_vanka", 0.0),
           ("M", 0.0), ("eta_st", -1.0), ("eps_mob", float("inf")), ("fuse_cells", -1),
           ("vanka_team_max", float("nan")), ("ch_team_max32", 2.0 ** 31),
           ("diverge_cycles", 0.5), ("step_time_limit", -1.0), ("precision", 3),
           ("precision", float("nan")), ("scheme", 0.5), ("coupled", float("nan"))]
    for key, value in bad:
        before = s.get_option(key)
        with pytest.raises(qn.QnschError) as e:
            s.set_option(key, value)
        assert e.value.code == -1, (key, value)
        assert s.get_option(key) == before, key
    for key, value in [("tol", 0.0), ("nu1", 0), ("maxcyc", 0), ("vanka_team_max", 2 ** 31 - 1),
                       ("omega_vanka", 1.5), ("step_time_limit", 0.25)]:
        s.set_option(key, value)
        assert s.get_option(key) == value, key


def test_time_step_must_be_positive_and_finite(qn):
    P = W.small_case()
    s = qn.Solver(**P.create_kwargs(), tol=P.tol)
    s.set_fields(P.fields())
    for dt in (0.0, -1e-3, float("inf"), float("nan")):
        with pytest.raises(qn.QnschError) as e:
            s.step(dt)
        assert e.value.code == -1, dt
        with pytest.raises(qn.QnschError) as e:
            s.begin_step(dt)
        assert e.value.code == -1, dt
    with pytest.raises(qn.QnschError) as e:
        qn.Batch([s]).step([float("inf")])
    assert e.value.code == -1
    s.step(P.dt)


def test_allocator_hook_and_an_injected_allocation_failure(qn):
    """Allocation faults injected on the host.  A handle created under a caller's
    allocator takes every block from it and gives every block back on destroy,
    with the same step result as cudaMalloc memory. It keeps that allocator
    after the hook is reset. An allocator that fails part way makes
    qnsch_create return QNSCH_ENOMEM, give back what it took and release its
    budget reservation."""
    import torch
    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
    live, state = {}, {"left": None, "allocs": 0}

    def alloc(nbytes, ctx):
        if state["left"] is not None:
            if state["left"] == 0:
                return None
            state["left"] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        live[p] = int(nbytes)
        state["allocs"] += 1
        return p

    def free(ptr, ctx):
        if live.pop(ptr, None) is not None:
            torch.cuda.caching_allocator_delete(ptr)

    a_cb, f_cb = ALLOC(alloc), FREE(free)
    L = qn.lib()
    P = W.small_case()
    ref = qn.Solver(**P.create_kwargs(), tol=P.tol)
    ref.set_fields(P.fields())
    ref.step(P.dt)
    gc.collect()
    _, u0 = qn.budget()
    try:
        assert L.qnsch_set_allocator(ctypes.cast(a_cb, ctypes.c_void_p),
                                     ctypes.cast(f_cb, ctypes.c_void_p), None) == 0
        s = qn.Solver(**P.create_kwargs(), tol=P.tol)
        assert L.qnsch_set_allocator(None, None, None) == 0  # s keeps its allocator
        s.set_fields(P.fields())
        s.step(P.dt)
        assert state["allocs"] > 0 and len(live) == state["allocs"]
        assert _same(s, ref)
        s.close()
        assert not live
        assert L.qnsch_set_allocator(ctypes.cast(a_cb, ctypes.c_void_p),
                                     ctypes.cast(f_cb, ctypes.c_void_p), None) == 0
        state["left"] = 2
        with pytest.raises(qn.QnschError) as e:
            qn.Solver(**P.create_kwargs(), tol=P.tol)
        assert e.value.code == -3
        assert not live and qn.budget()[1] == u0
    finally:
        L.qnsch_set_allocator(None, None, None)


def test_batch_refuses_members_that_came_to_share_a_stream(qn):
    import torch
    P = W.small_case()
    a, b = _pair(qn, P)
    B = qn.Batch([a, b])
    st = torch.cuda.Stream()
    a.set_stream(st)
    b.set_stream(st)
    with pytest.raises(qn.QnschError) as e:
        B.step([P.dt, P.dt])
    assert e.value.code == -1
    a.set_stream(None)
    b.set_stream(None)
    status, _ = B.step([P.dt, P.dt])
    assert status == [0, 0] and _same(a, b)
