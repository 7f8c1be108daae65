"""The skewed-chunk schedule of the error-equation smoothers (k_skew, option
skew_cells32): the passes of nu smoothing steps (CH red, CH black and the
Vanka colours, or the coupled colours) run over chunks of skew_rows rows, pass
p trailing pass p - 1 by a chunk and two rows, one launch per diagonal.  Every
visit sees the values it sees when each pass is a launch over the whole level
and runs the same device code, so against per-colour launches with one lane
per visit the V-cycle counts, residuals and fields are bit-identical: walls
and periodic x (5 and 8 colours), a ragged grid, chunks of one row, of a few
rows and taller than the level, the coupled block, FP32 and FP64 error
levels, and the Rayleigh-Taylor workload at its full 1024 x 4096 size with the
library's default thresholds.  With the schedule on, the mixed step matches
the FP64 oracle within the mixed-precision bars, and its launches are timed as
profiling kind 5."""
import numpy as np
import pytest

from mixed_tol import MIXED_TOL
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# per-colour launches with one lane per visit, as k_skew runs them
SINGLE = {"vanka_team_max32": 0, "ch_team_max32": 0}


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


CASES = [
    ("walls_sep", W.small_case(64, 96, False, rho_ratio=10.0), {"precision": 1}),
    ("periodic_sep", W.small_case(64, 64, True, rho_ratio=10.0), {"precision": 1}),
    ("ragged", W.small_case(48, 72, False), {"precision": 1}),
    ("coupled_walls", W.small_case(64, 96, False, rho_ratio=10.0), {"precision": 1, "coupled": 1}),
    ("coupled_periodic", W.small_case(96, 64, True), {"precision": 1, "coupled": 1}),
    ("fp64_error_form", W.small_case(64, 96, False), {"precision": 2}),
]


def _same(a, b, P, steps):
    f = P.fields()
    a.set_fields(f)
    b.set_fields(f)
    for _ in range(steps):
        na, ra = a.step(P.dt)
        nb, rb = b.step(P.dt)
        assert na == nb and ra == rb, (na, nb, ra, rb)
    fa, fb = a.get_fields(), b.get_fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("rows", [1, 5, 40])
@pytest.mark.parametrize("name,P,opts", CASES, ids=[c[0] for c in CASES])
def test_skew_equals_per_colour_launches(qn, name, P, opts, rows):
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, skew_cells32=1, skew_rows=rows, **SINGLE, **opts)
    b = qn.Solver(**P.create_kwargs(), tol=P.tol, skew_cells32=0, **SINGLE, **opts)
    _same(a, b, P, 2)


def test_skew_equals_per_colour_launches_at_full_size(qn):
    """Rayleigh-Taylor 1024 x 4096, mixed precision: the schedule on the two
    finest levels (the levels below keep their per-colour team launches)."""
    P = W.rayleigh_taylor_1024x4096()
    a = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, skew_cells32=1 << 20, skew_rows=64)
    b = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1)
    _same(a, b, P, 1)


def test_skew_launches_are_timed_as_kind_5(qn):
    P = W.small_case(64, 96, False)
    s = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, skew_cells32=1 << 12)
    s.set_fields(P.fields())
    l0 = qn.kernel_launches()
    s.profile(1 << 5)
    n, _ = s.step(P.dt)
    launches, ms, visits = s.profile_read_kind("skew")
    s.profile(False)
    assert qn.kernel_launches() > l0
    # one bracket per smoothing block of the finest level: nu1 + nu2 steps per cycle
    assert launches == 2 * n and ms > 0.0
    assert visits == 64 * 96 * 4 * n
    assert s.profile_read_kind("vanka_finest")[0] == 0


def test_skew_mixed_step_matches_the_oracle(qn):
    from oracle.ref import RefSolver
    P = W.small_case(64, 96, False, rho_ratio=10.0)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, skew_cells32=1, skew_rows=8)
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
