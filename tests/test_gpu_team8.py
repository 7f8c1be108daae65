"""Eight lanes per FP64 Vanka block (option vanka_team8_max): each lane pair
evaluates one momentum row's residual in two halves that one shuffle adds, so
the visit's result is that of the four-lane and single-lane visits up to the
order of two additions.  Against the FP64 oracle: single colour sweeps at
1e-11 (walls, periodic, ragged, the smallest grids), V-cycles with the
per-level and the single-block coarse launches at 1e-10, and a full step of
the 256x512 droplet with equal V-cycle counts at 1e-10."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KW = dict(Lx=1.0, levels=0, rho1=1.0, rho2=3.0, eta1=1.0, eta2=2.5, Re=50.0, We=5.0, Pe=20.0,
          Cn=0.05, Fr=0.8)
BIG = 1 << 30


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


@pytest.mark.parametrize("m1,m2,px", [(16, 12, False), (16, 12, True), (37, 29, False),
                                     (40, 24, True), (2, 2, False), (8, 4, True)])
def test_team8_sweep_parity(qn, m1, m2, px):
    g = qn.Solver(m1, m2, periodic_x=px, vanka_team8_max=BIG, **KW)
    r = RefSolver(m1, m2, periodic_x=px, **KW)
    fn = W.random_state(m1, m2, px, seed=27)
    fx = W.random_state(m1, m2, px, seed=28)
    for s in (g, r):
        s.set_fields(fn)
        s.begin_step(2e-3)
        s.set_iterate(fx)
    for colour in range(g.ncolours_vanka):
        g.smooth_vanka(colour)
        r.smooth_vanka(colour)
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-11, (colour, k)


@pytest.mark.parametrize("m1,m2,px,fuse", [(32, 48, False, 128), (40, 40, True, 128),
                                           (32, 48, False, 0), (64, 96, True, 128)])
def test_team8_vcycle_parity(qn, m1, m2, px, fuse):
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs(), vanka_team8_max=BIG, fuse_cells=fuse)
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


def test_team8_full_step_rising_drop(qn):
    P = W.rising_drop_256x512()
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, vanka_team8_max=2048)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    ng, _ = g.step(P.dt)
    nr, _ = r.step(P.dt)
    assert ng == nr
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        assert relerr(fg[k], fr[k]) <= 1e-10, k
