"""The banded wavefront smoother (k_wave, option wave_cells32): nu smoothing
steps on an error-equation level as one launch whose passes (CH red/black and
the Vanka or coupled colours) run band by band in a skewed order.  Every visit
sees the values it sees when each pass is a launch over the whole level, and
runs the same device code, so a step with the wavefront gives the results of
the per-colour launches up to rounding (the compiler may contract a
multiply-add differently inside the two kernels): the same V-cycle counts and
fields within 1e-12, on wall-bounded and periodic grids (5 and 8 colours),
ragged sizes, band heights that do and do not divide the rows, single-lane and
four-lane blocks, the coupled block, FP32 and FP64 error levels.  With the
wavefront on, the mixed step still matches the FP64 oracle within the
mixed-precision bars.  The bounded wait: a test hook makes one
wait wait for a count nothing reaches; the wait runs out, the step ends with
QNSCH_ETIMEOUT without committing, and the handle steps normally afterwards."""
import numpy as np
import pytest

from mixed_tol import MIXED_TOL
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
    # name, problem, options of both solvers, wavefront options
    ("walls_sep", W.small_case(64, 96, False, rho_ratio=10.0), {"precision": 1}, {"wave_rows": 8}),
    ("periodic_sep", W.small_case(64, 64, True, rho_ratio=10.0), {"precision": 1},
     {"wave_rows": 4}),
    ("ragged_rows", W.small_case(48, 72, False), {"precision": 1}, {"wave_rows": 5}),
    ("single_lane", W.small_case(64, 96, True), {"precision": 1, "vanka_team_max32": 0},
     {"wave_rows": 8}),
    ("ch_teams", W.small_case(64, 64, False), {"precision": 1, "ch_team_max32": 1 << 20},
     {"wave_rows": 6}),
    ("coupled", W.small_case(64, 96, False, rho_ratio=10.0), {"precision": 1, "coupled": 1},
     {"wave_rows": 8}),
    ("coupled_single", W.small_case(96, 64, True), {"precision": 1, "coupled": 1,
                                                     "vanka_team_max32": 0}, {"wave_rows": 4}),
    ("fp64_error_form", W.small_case(64, 96, False), {"precision": 2}, {"wave_rows": 8}),
    ("drop_256x512", W.rising_drop_256x512(), {"precision": 1}, {"wave_rows": 8}),
]


@pytest.mark.parametrize("name,P,opts,wopts", CASES, ids=[c[0] for c in CASES])
def test_wavefront_step_matches_per_colour_launches(qn, name, P, opts, wopts):
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, wave_cells32=1, **opts, **wopts)
    b = qn.Solver(**P.create_kwargs(), tol=P.tol, wave_cells32=0, **opts)
    f = P.fields()
    a.set_fields(f)
    b.set_fields(f)
    for _ in range(2):
        na, ra = a.step(P.dt)
        nb, rb = b.step(P.dt)
        assert na == nb, (na, nb, ra, rb)
        assert abs(ra - rb) <= 1e-6 * rb, (ra, rb)
    fa, fb = a.get_fields(), b.get_fields()
    for k in fa:
        e = np.max(np.abs(fa[k] - fb[k])) / max(np.max(np.abs(fb[k])), 1e-300)
        assert e <= 1e-12, (k, e)


def test_wavefront_counts_as_its_own_kind_and_runs(qn):
    """The wavefront launches are the ones timed as kind 4, one per smoothing
    block of a level, each with the cell visits of its steps."""
    P = W.small_case(64, 96, False)
    s = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, wave_cells32=1)
    s.set_fields(P.fields())
    s.profile(1 << 4)
    n, _ = s.step(P.dt)
    launches, ms, visits = s.profile_read_kind(4)
    s.profile(False)
    assert launches > 0 and ms > 0.0 and visits > 0.0
    assert visits >= launches * 8 * 8 * 2  # at least nu = 2 steps over an 8 x 8 level


@pytest.mark.parametrize("device_loop", [1, 0])
def test_a_wait_that_runs_out_ends_the_step_with_etimeout(qn, device_loop):
    P = W.small_case(64, 96, False)
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, wave_cells32=1,
                  device_loop=device_loop)
    b = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, wave_cells32=1,
                  device_loop=device_loop)
    a.set_fields(P.fields())
    b.set_fields(P.fields())
    f0 = a.get_fields()
    a.set_option("wave_stall", 1)
    a.set_option("wave_wait_cycles", 2000000)
    with pytest.raises(qn.QnschError) as e:
        a.step(P.dt)
    assert e.value.code == -6
    f1 = a.get_fields()
    assert all(np.array_equal(f0[k], f1[k]) for k in f0)
    # the hook off again: the handle steps as an untouched one does
    a.set_option("wave_stall", 0)
    a.set_option("wave_wait_cycles", 1 << 31)
    na, _ = a.step(P.dt)
    nb, _ = b.step(P.dt)
    fa, fb = a.get_fields(), b.get_fields()
    assert na == nb and all(np.array_equal(fa[k], fb[k]) for k in fa)


def test_wavefront_mixed_step_matches_the_oracle(qn):
    from oracle.ref import RefSolver
    P = W.small_case(64, 96, False, rho_ratio=10.0)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, wave_cells32=1)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(2):
        ng, rg = g.step(P.dt)
        nr, rr = r.step(P.dt)
        assert rg <= P.tol and rr <= P.tol
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        err = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
        assert err <= MIXED_TOL[k], (k, err)
