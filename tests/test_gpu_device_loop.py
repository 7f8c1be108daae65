"""The outer-cycle loop on the device: one qnsch_step is one CUDA graph (the
initial residual, a conditional WHILE node around the outer cycle, a
conditional IF node around the commit, one copy of the results to the host),
option device_loop = 1.

Against the host-driven loop (device_loop = 0, the default: the host reads
the norms after every cycle and queues the next), on the same inputs: the same
V-cycle counts, bit-identical fields and the same mass, for the FP64 path,
mixed precision with either smoother, and the projection method.  The
handle keeps device_loop = 1 after its steps, so the graph was built and ran.
Each step launches exactly 2 + k more kernels than the host-driven step of
k cycles (the start-time and loop-control kernels), which pins the launch
count the library reports for graph replays."""
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


CASES = [
    ("fp64", W.small_case(32, 32, True), {}),
    ("fp64_walls", W.small_case(48, 64, False, rho_ratio=10.0), {}),
    ("mixed", W.small_case(64, 48, False, rho_ratio=10.0), {"precision": 1}),
    ("mixed_coupled", W.small_case(64, 64, True, rho_ratio=10.0), {"precision": 1, "coupled": 1}),
    ("projection", W.small_case(32, 64, False), {"scheme": 1}),
]


@pytest.mark.parametrize("name,P,opts", CASES, ids=[c[0] for c in CASES])
def test_device_loop_equals_host_loop(qn, name, P, opts):
    dev = qn.Solver(**P.create_kwargs(), tol=P.tol, device_loop=1, **opts)
    host = qn.Solver(**P.create_kwargs(), tol=P.tol, device_loop=0, **opts)
    f = P.fields()
    dev.set_fields(f)
    host.set_fields(f)
    for _ in range(3):
        l0 = qn.kernel_launches()
        nd, rd = dev.step(P.dt)
        l1 = qn.kernel_launches()
        nh, rh = host.step(P.dt)
        l2 = qn.kernel_launches()
        assert nd == nh, (nd, nh)
        assert rd == rh, (rd, rh)
        assert (l1 - l0) - (l2 - l1) == 2 + nd, (l1 - l0, l2 - l1, nd)
    fd, fh = dev.get_fields(), host.get_fields()
    for k in fd:
        assert np.array_equal(fd[k], fh[k]), k
    assert dev.mass() == host.mass()
    assert dev.energy() == host.energy()
    assert dev.get_option("device_loop") == 1.0


def test_device_loop_step_that_does_not_converge_is_not_committed(qn):
    """maxcyc = 1 at an unreachable tolerance: QNSCH_ENOTCONV after one cycle
    with the committed state untouched, in both loops alike."""
    P = W.small_case()
    out = []
    for loop in (1, 0):
        s = qn.Solver(**P.create_kwargs(), tol=1e-15, maxcyc=1, device_loop=loop)
        s.set_fields(P.fields())
        f0 = s.get_fields()
        with pytest.raises(qn.QnschError) as e:
            s.step(P.dt)
        assert e.value.code == -4
        f1 = s.get_fields()
        assert all(np.array_equal(f0[k], f1[k]) for k in f0)
        out.append(s)
    # both handles stay usable and agree once the tolerance is reachable
    for s in out:
        s.set_option("tol", P.tol)
        s.set_option("maxcyc", 50)
    na, _ = out[0].step(P.dt)
    nb, _ = out[1].step(P.dt)
    assert na == nb
    fa, fb = out[0].get_fields(), out[1].get_fields()
    assert all(np.array_equal(fa[k], fb[k]) for k in fa)


def test_batch_of_device_loops_equals_alone(qn):
    """Members whose device_loop is on step in a batch through the batch's
    host-driven state machine: each member's result equals its host-driven
    step alone."""
    probs = [W.small_case(32, 32, True), W.small_case(64, 48, False, rho_ratio=10.0),
             W.capillary_64()]
    batch, alone = [], []
    for P in probs:
        b = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, coupled=1, device_loop=1)
        a = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, coupled=1, device_loop=0)
        b.set_fields(P.fields())
        a.set_fields(P.fields())
        batch.append(b)
        alone.append(a)
    B = qn.Batch(batch)
    for _ in range(2):
        st, cyc = B.step([P.dt for P in probs])
        assert st == [0, 0, 0], st
        for a, P, n in zip(alone, probs, cyc):
            na, _ = a.step(P.dt)
            assert na == n
    for a, b in zip(alone, batch):
        fa, fb = a.get_fields(), b.get_fields()
        assert all(np.array_equal(fa[k], fb[k]) for k in fa)


@pytest.mark.parametrize("device_loop", [0, 1])
def test_async_step_equals_step(qn, device_loop):
    """qnsch_step_launch + qnsch_step_poll give what qnsch_step gives: the same
    cycles, residual, status and bit-identical fields, with the host-driven
    loop advanced by the polls and with the step graph; the handle refuses a
    second launch or a plain step while one is in flight, and a poll without
    a launch."""
    P = W.small_case(48, 64, False, rho_ratio=10.0)
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, coupled=1,
                  device_loop=device_loop)
    b = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, coupled=1)
    a.set_fields(P.fields())
    b.set_fields(P.fields())
    with pytest.raises(qn.QnschError) as e:
        a.step_poll()
    assert e.value.code == -8
    for _ in range(2):
        a.step_launch(P.dt)
        with pytest.raises(qn.QnschError) as e:
            a.step_launch(P.dt)
        assert e.value.code == -8
        with pytest.raises(qn.QnschError) as e:
            a.step(P.dt)
        assert e.value.code == -8
        out = None
        while out is None:
            out = a.step_poll()
        na, ra, st, ms = out
        nb, rb = b.step(P.dt)
        assert st == 0 and na == nb and ra == rb and ms > 0.0
    fa, fb = a.get_fields(), b.get_fields()
    assert all(np.array_equal(fa[k], fb[k]) for k in fa)
