"""Projection method (Sec. 6.2, solver Sec. 7.2) on the GPU against the oracle:
residuals and single sweeps from random states, V-cycles from physical states
(walls and periodic, several tiles and ragged tails), full steps (cycle counts,
fields, mass, energy and dissipation), and the full-size droplet step."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def same_fields(fg, fr, tol, keys=("c", "mu", "p", "u", "v")):
    for k in keys:
        scale = max(np.max(np.abs(fr[k])), 1e-30)
        err = np.max(np.abs(fg[k] - fr[k])) / scale
        assert err <= tol, (k, err)


def _pair(qn, P, **opt):
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, scheme=1, **opt)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, scheme=1, **opt)
    return g, r


@pytest.mark.parametrize("m1,m2,px", [(37, 29, False), (32, 24, True), (14, 6, True)])
def test_projection_residual_and_sweep_parity(qn, m1, m2, px):
    P = W.small_case(m1, m2, px)
    g, r = _pair(qn, P)
    f = W.random_state(m1, m2, px, seed=5)
    for s in (g, r):
        s.set_fields(f)
        s.begin_step(2e-3)
        s.set_iterate(W.random_state(m1, m2, px, seed=55, scale=dict(u=0.02, v=0.02, p=0.05)))
    rg, ng = g.residual()
    rr, nr = r.residual()
    same_fields(rg, rr, 1e-12)
    g.smooth(1)
    r.smooth(1)
    same_fields(g.get_iterate(), r.get_iterate(), 1e-10)


@pytest.mark.parametrize("m1,m2,px", [(32, 48, False), (32, 48, True), (24, 40, False),
                                     (40, 40, True), (64, 256, True)])
def test_projection_vcycle_parity(qn, m1, m2, px):
    P = W.small_case(m1, m2, px)
    g, r = _pair(qn, P)
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    assert g.levels == r.levels
    for _ in range(3):
        ng = g.vcycle()
        nr = r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-10)
        assert np.allclose(ng, nr, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("px", [False, True])
def test_projection_full_steps_parity(qn, px):
    P = W.small_case(32, 48, px, rho_ratio=10.0)
    g, r = _pair(qn, P)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    for _ in range(3):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert ng == nr and resg <= P.tol
    same_fields(g.get_fields(), r.get_fields(), 1e-10)
    mg, mr = g.mass(), r.mass()
    assert abs(mg[0] - mr[0]) <= 1e-13 * mr[0] and abs(mg[1] - mr[1]) <= 1e-13 * mr[1]
    eg, dg = g.energy()
    assert abs(eg - r.energy()) <= 1e-12 * abs(r.energy()) and dg > 0


def test_projection_dissipation_matches_oracle(qn):
    """The last step's dissipation (viscous, CH and the two kinetic terms of the
    projection method) equals the oracle's for the same step."""
    P = W.small_case(32, 32, True, rho_ratio=5.0)
    g, r = _pair(qn, P)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    g.step(P.dt)
    r.begin_step(P.dt)
    while max(r.vcycle()[:5]) > P.tol:
        pass
    d_oracle = r.iterate_dissipation()
    _, d_gpu = g.energy()
    assert abs(d_gpu - d_oracle) <= 1e-8 * abs(d_oracle)


def test_projection_full_size_droplet_step(qn):
    """The bench droplet (256x512, walls, 8 levels) by the projection method:
    same cycle count and fields as the oracle after one step."""
    P = W.rising_drop_256x512()
    g, r = _pair(qn, P)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    ng, resg = g.step(P.dt)
    nr, resr = r.step(P.dt)
    assert ng == nr and resg <= P.tol
    same_fields(g.get_fields(), r.get_fields(), 1e-10)


def test_projection_option_rules(qn):
    g = qn.Solver(16, 16, scheme=1)
    for key, val in (("coupled", 1), ("precision", 1)):
        with pytest.raises(qn.QnschError):
            g.set_option(key, val)
    h = qn.Solver(16, 16, precision=1)
    with pytest.raises(qn.QnschError):
        h.set_option("scheme", 1)


@pytest.mark.parametrize("px", [False, True])
def test_projection_fused_coarse_levels_match_per_level_launches(qn, px):
    """The single-block V-cycle of the small levels runs the projection
    smoother in the same colour order as the per-level launches."""
    P = W.small_case(64, 96, px)
    out = []
    for fuse in (0, 10 ** 6):
        g = qn.Solver(**P.create_kwargs(), scheme=1, fuse_cells=fuse)
        g.set_fields(P.fields())
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[0], out[1], 1e-12)


@pytest.mark.parametrize("px", [False, True])
def test_projection_team_launches_match_single_lane(qn, px):
    """The 4x4 intermediate-velocity blocks (vanka_team_max), the CH Newton
    steps and the pressure Gauss-Seidel (ch_team_max) with four lanes per
    block or cell do the arithmetic of one lane, with face terms summed in
    another order and the block solve split over the lanes: after two
    V-cycles the iterates agree within the 1e-10 parity bar."""
    P = W.small_case(128, 192, px)
    out = []
    for tm in (0, 10 ** 9):
        g = qn.Solver(**P.create_kwargs(), scheme=1, vanka_team_max=tm, ch_team_max=tm,
                      fuse_cells=0)
        g.set_fields(P.fields())
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[0], out[1], 1e-10)
