"""The predicted initial iterate (option "predictor") on the GPU against the
oracle with the same option: the same V-cycle counts and every field within
1e-10 over several steps, constant and changing step sizes, the paper's
smoother, the coupled block and the projection method, the 256x512 drop at the
bench's smoothing counts; mixed precision within the mixed bars.  The history
round trip makes a resumed run repeat the uninterrupted one bit for bit (also
through a checkpoint file), and the step graph (device_loop), asynchronous
steps and batches give what the host-driven step gives as the predictor's
weights change from step to step."""
import numpy as np
import pytest

from mixed_tol import check_mixed
from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def _dts(P, n, vary):
    return [P.dt * (1.0 + (0.3 * ((k % 3) - 1) if vary else 0.0)) for k in range(n)]


CASES = [
    ("walls_linear", W.small_case(32, 48, False), {"predictor": 1}, False),
    ("walls_quadratic_varying_dt", W.small_case(32, 48, False), {"predictor": 2}, True),
    ("periodic_quadratic", W.small_case(32, 32, True), {"predictor": 2}, False),
    ("coupled_quadratic", W.small_case(32, 48, False), {"predictor": 2, "coupled": 1}, True),
    ("projection_quadratic", W.small_case(32, 64, False), {"predictor": 2, "scheme": 1}, False),
    ("capillary_quadratic", W.capillary_64(), {"predictor": 2, "nu1": 3, "nu2": 2}, False),
]


@pytest.mark.parametrize("name,P,opts,vary", CASES, ids=[c[0] for c in CASES])
def test_predictor_matches_the_oracle(qn, name, P, opts, vary):
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for dt in _dts(P, 6, vary):
        ng, rg = g.step(dt)
        nr, rr = r.step(dt)
        assert ng == nr and rg <= P.tol and rr <= P.tol, (ng, nr)
    assert g.get_option("history") == r.get_option("history") == 2
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        e = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
        assert e <= 1e-10, (k, e)


def test_predictor_full_size_at_the_bench_counts(qn):
    P = W.rising_drop_256x512()
    opts = {"predictor": 2, "nu1": 3, "nu2": 2}
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(4):
        ng, _ = g.step(P.dt)
        nr, _ = r.step(P.dt)
        assert ng == nr
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        e = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
        assert e <= 1e-10, (k, e)


def test_mixed_predictor_within_the_bars(qn):
    P = W.small_case(64, 48, False, rho_ratio=10.0)
    opts = {"predictor": 2, "coupled": 1, "nu1": 1, "nu2": 2}
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(5):
        ng, _ = g.step(P.dt)
        nr, _ = r.step(P.dt)
        assert abs(ng - nr) <= 1
    check_mixed(g.get_fields(), r.get_fields())


def _run(qn, P, opts, n, start=None, hist=()):
    s = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    s.set_fields(P.fields() if start is None else start)
    for k, (f, dt) in enumerate(hist):
        s.set_history(k, f, dt)
    cyc = [s.step(P.dt)[0] for _ in range(n)]
    return s, cyc


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_with_history_repeats_the_run(qn, tmp_path, precision):
    P = W.small_case(32, 48, False)
    opts = {"predictor": 2, "precision": precision}
    full, cyc_full = _run(qn, P, opts, 6)
    half, cyc_a = _run(qn, P, opts, 3)
    hist = [half.history(k) for k in range(int(half.get_option("history")))]
    assert len(hist) == 2
    rest, cyc_b = _run(qn, P, opts, 3, start=half.get_fields(), hist=hist)
    assert cyc_a + cyc_b == cyc_full
    ff, fr = full.get_fields(), rest.get_fields()
    assert all(np.array_equal(ff[k], fr[k]) for k in ff)
    # the same through a checkpoint file
    path = str(tmp_path / "ck.npz")
    half.save_checkpoint(path, t=3 * P.dt, n=3)
    again, t, n = qn.Solver.from_checkpoint(path)
    assert n == 3 and again.get_option("history") == 2
    cyc_c = [again.step(P.dt)[0] for _ in range(3)]
    assert cyc_c == cyc_b
    fa = again.get_fields()
    assert all(np.array_equal(ff[k], fa[k]) for k in ff)


def test_device_loop_async_and_batch_equal_the_host_step(qn):
    """As the history fills (weights (1,0,0), then linear, then quadratic) and
    when dt changes, the step graph is rebuilt and gives the host-driven
    step's counts and bits; so do step_launch/step_poll and a batch."""
    P = W.small_case(32, 48, False)
    opts = {"predictor": 2}
    dts = [P.dt, P.dt, P.dt, 1.3 * P.dt, 1.3 * P.dt, P.dt]
    host = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    dev = qn.Solver(**P.create_kwargs(), tol=P.tol, device_loop=1, **opts)
    asy = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    bat = qn.Solver(**P.create_kwargs(), tol=P.tol, **opts)
    for s in (host, dev, asy, bat):
        s.set_fields(P.fields())
    B = qn.Batch([bat])
    for dt in dts:
        nh, rh = host.step(dt)
        nd, rd = dev.step(dt)
        asy.step_launch(dt)
        out = None
        while out is None:
            out = asy.step_poll()
        st, cy = B.step([dt])
        assert (nd, rd) == (nh, rh)
        assert out[0] == nh and out[1] == rh and out[2] == 0
        assert st == [0] and cy == [nh]
    assert dev.get_option("device_loop") == 1.0
    fh = host.get_fields()
    for s in (dev, asy, bat):
        f = s.get_fields()
        assert all(np.array_equal(fh[k], f[k]) for k in fh)


def test_a_failed_step_keeps_the_history(qn):
    P = W.small_case(32, 32, True)
    s = qn.Solver(**P.create_kwargs(), tol=P.tol, predictor=2)
    s.set_fields(P.fields())
    for _ in range(3):
        s.step(P.dt)
    h0 = s.history(0)[0]
    s.set_option("maxcyc", 1)
    s.set_option("tol", 1e-15)
    with pytest.raises(qn.QnschError):
        s.step(P.dt)
    assert s.get_option("history") == 2
    assert np.array_equal(s.history(0)[0]["c"], h0["c"])
    s.set_fields(P.fields())
    assert s.get_option("history") == 0
