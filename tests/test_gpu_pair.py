"""A lane pair per FP64 Vanka block (option vanka_pair_max): the x pair of rows
on one lane, the y pair on the other, each lane factoring its own 2x2 block of
the structured solve; sums associated as in the four-lane team.  Against the
FP64 oracle: single colour sweeps at 1e-11 (walls, periodic, ragged, the
smallest grids), V-cycles with the pairs on every per-level launch at 1e-10,
and full steps of the 256x512 droplet with equal V-cycle counts at 1e-10;
against the four-lane team on the same sweep, agreement to rounding.  The
split launch (option vanka_split: one lane per block for the first slots of a
colour, pairs for the rest) is held to the same bars."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(Lx=1.0, levels=0, rho1=1.0, rho2=3.0, eta1=1.0, eta2=2.5, Re=50.0, We=5.0, Pe=20.0,
          Cn=0.05, Fr=0.8)
BIG = 1 << 30
# every per-level launch with pairs: no four-lane teams, pairs up to any size
PAIRS = dict(vanka_team_max=0, vanka_pair_max=BIG)


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _begin(s, fn, fx):
    s.set_fields(fn)
    s.begin_step(2e-3)
    s.set_iterate(fx)


@pytest.mark.parametrize("m1,m2,px", [(16, 12, False), (16, 12, True), (37, 29, False),
                                     (40, 24, True), (2, 2, False), (8, 4, True), (65, 33, False)])
def test_pair_sweep_parity(qn, m1, m2, px):
    g = qn.Solver(m1, m2, periodic_x=px, **PAIRS, **KW)
    assert g.get_option("vanka_pair_max") == BIG
    r = RefSolver(m1, m2, periodic_x=px, **KW)
    fn = W.random_state(m1, m2, px, seed=37)
    fx = W.random_state(m1, m2, px, seed=38)
    for s in (g, r):
        _begin(s, fn, fx)
    for colour in range(g.ncolours_vanka):
        g.smooth_vanka(colour)
        r.smooth_vanka(colour)
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-11, (colour, k)


@pytest.mark.parametrize("m1,m2,px", [(37, 29, False), (40, 24, True)])
def test_pair_matches_four_lane_team(qn, m1, m2, px):
    """Same sweep with pairs and with four-lane teams: the team's arithmetic,
    so the fields agree to rounding (the compiler may contract differently)."""
    a = qn.Solver(m1, m2, periodic_x=px, **PAIRS, **KW)
    b = qn.Solver(m1, m2, periodic_x=px, vanka_team_max=BIG, **KW)
    fn = W.random_state(m1, m2, px, seed=41)
    fx = W.random_state(m1, m2, px, seed=42)
    for s in (a, b):
        _begin(s, fn, fx)
        for colour in range(s.ncolours_vanka):
            s.smooth_vanka(colour)
    fa, fb = a.get_iterate(), b.get_iterate()
    for k in fa:
        assert relerr(fa[k], fb[k]) <= 1e-13, k


@pytest.mark.parametrize("m1,m2,px,fuse", [(32, 48, False, 128), (40, 40, True, 128),
                                           (32, 48, False, 0), (64, 96, True, 128)])
def test_pair_vcycle_parity(qn, m1, m2, px, fuse):
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs(), fuse_cells=fuse, **PAIRS)
    r = RefSolver(**P.create_kwargs())
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        g.vcycle()
        r.vcycle()
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-10, k


def test_pair_full_steps_rising_drop(qn):
    """Two steps of the 256x512 droplet with pairs on the finest level (the
    levels below keep their four-lane teams) and the headline's smoothing
    counts and predictor: equal V-cycle counts and fields within 1e-10."""
    P = W.rising_drop_256x512()
    opts = dict(nu1=1, nu2=1, nu1_fine=2, nu2_fine=3, predictor=2)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, vanka_pair_max=1 << 20, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(2):
        ng, _ = g.step(P.dt)
        nr, _ = r.step(P.dt)
        assert ng == nr
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        assert relerr(fg[k], fr[k]) <= 1e-10, k


# ---- the split launch (option vanka_split): one lane per block for the first
# slots of a colour, lane pairs for the rest


@pytest.mark.parametrize("m1,m2,px,split", [(37, 29, False, 64), (40, 24, True, 32),
                                           (65, 33, False, 96), (16, 12, True, 2)])
def test_split_sweep_parity(qn, m1, m2, px, split):
    """A forced split (split slots one lane each, rounded down to a multiple
    of 32; 2 rounds to none, so every block is a pair) against the oracle."""
    g = qn.Solver(m1, m2, periodic_x=px, vanka_team_max=0, vanka_split=split, **KW)
    r = RefSolver(m1, m2, periodic_x=px, **KW)
    fn = W.random_state(m1, m2, px, seed=47)
    fx = W.random_state(m1, m2, px, seed=48)
    for s in (g, r):
        _begin(s, fn, fx)
    for colour in range(g.ncolours_vanka):
        g.smooth_vanka(colour)
        r.smooth_vanka(colour)
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-11, (colour, k)


def test_split_vcycle_parity(qn):
    P = W.small_case(64, 96, True)
    g = qn.Solver(**P.create_kwargs(), vanka_team_max=0, vanka_split=64)
    r = RefSolver(**P.create_kwargs())
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        g.vcycle()
        r.vcycle()
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-10, k


def test_split_full_steps_rising_drop(qn):
    """The cost model's split (vanka_split = 1) on the 256x512 droplet, whose
    finest colours (26,214 blocks) fill a GB300's 608 sub-partitions 1.35
    times: three steps with the headline's options, equal V-cycle counts and
    fields within 1e-10 of the oracle."""
    P = W.rising_drop_256x512()
    opts = dict(nu1=1, nu2=1, nu1_fine=2, nu2_fine=3, predictor=2)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, vanka_split=1, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(3):
        ng, _ = g.step(P.dt)
        nr, _ = r.step(P.dt)
        assert ng == nr
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        assert relerr(fg[k], fr[k]) <= 1e-10, k
