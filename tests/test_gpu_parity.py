"""Parity of the CUDA path (libqnsch.so, through its C ABI) with the FP64 oracle.

Element-by-element comparisons on the same seeded inputs: the residual of every
family, single colour sweeps of both smoothers, a full smoothing step, one
V-cycle, and full time steps; conservation and energy checks on the GPU
results; edge cases (smallest grids, ragged sizes, periodic seams) and error
statuses.  FP64 tolerances: per-kernel results to 1e-11 relative (rounding
order and FMA contraction differ between the two builds), converged steps to
1e-10 relative in max norm per field.  Mixed precision: the per-field bars of
tests/mixed_tol.py.
"""
import math

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


KW = dict(Lx=1.0, levels=0, rho1=1.0, rho2=3.0, eta1=1.0, eta2=2.5, Re=50.0, We=5.0, Pe=20.0,
          Cn=0.05, Fr=0.8)


def pair(qn, m1, m2, px, **over):
    kw = dict(KW, **over)
    return qn.Solver(m1, m2, periodic_x=px, **kw), RefSolver(m1, m2, periodic_x=px, **kw)


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def load_random(g, r, px, seed=7, dt=2e-3):
    fn = W.random_state(g.m1, g.m2, px, seed=seed)
    fx = W.random_state(g.m1, g.m2, px, seed=seed + 1)
    for s in (g, r):
        s.set_fields(fn)
        s.begin_step(dt)
        s.set_iterate(fx)
    return fn, fx


def same_fields(fg, fr, tol, keys=("c", "mu", "p", "u", "v")):
    for k in keys:
        e = relerr(fg[k], fr[k])
        assert e <= tol, (k, e)


SIZES = [(16, 12, False), (16, 12, True), (37, 29, False), (40, 24, True), (2, 2, False),
         (4, 6, True), (70, 45, False), (10, 8, True), (14, 6, True)]


@pytest.mark.parametrize("m1,m2,px", SIZES)
def test_residual_parity(qn, m1, m2, px):
    g, r = pair(qn, m1, m2, px)
    load_random(g, r, px)
    rg, ng = g.residual()
    rr, nr = r.residual()
    for k in rg:
        sl = (slice(None), slice(1, m1 + (1 if px else 0))) if k == "u" else (
            (slice(1, m2), slice(None)) if k == "v" else (slice(None), slice(None)))
        assert relerr(rg[k][sl], rr[k][sl]) <= 1e-11, k
    assert np.allclose(ng, nr, rtol=1e-11, atol=0)


@pytest.mark.parametrize("m1,m2,px", SIZES)
def test_ch_sweep_parity(qn, m1, m2, px):
    g, r = pair(qn, m1, m2, px)
    load_random(g, r, px, seed=17)
    for colour in (0, 1):
        g.smooth_ch(colour)
        r.smooth_ch(colour)
        same_fields(g.get_iterate(), r.get_iterate(), 1e-11)


@pytest.mark.parametrize("m1,m2,px", SIZES)
def test_vanka_sweep_parity(qn, m1, m2, px):
    g, r = pair(qn, m1, m2, px)
    load_random(g, r, px, seed=27)
    for colour in range(g.ncolours_vanka):
        g.smooth_vanka(colour)
        r.smooth_vanka(colour)
        same_fields(g.get_iterate(), r.get_iterate(), 1e-11)


@pytest.mark.parametrize("m1,m2,px", [(32, 24, False), (32, 24, True)])
def test_smoothing_parity_random_state(qn, m1, m2, px):
    g, r = pair(qn, m1, m2, px)
    load_random(g, r, px, seed=37)
    g.smooth(2)
    r.smooth(2)
    same_fields(g.get_iterate(), r.get_iterate(), 1e-10)


@pytest.mark.parametrize("m1,m2,px", [(32, 48, False), (32, 48, True), (24, 40, False),
                                     (40, 40, True), (56, 56, True)])
def test_vcycle_parity_from_physical_state(qn, m1, m2, px):
    """V-cycles (all levels, transfers, coarsest solve, gauge) from the level-n state."""
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs())
    r = RefSolver(**P.create_kwargs())
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    assert g.levels == r.levels
    for _ in range(3):
        ng = g.vcycle()
        nr = r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-10)
        assert np.allclose(ng, nr, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("coupled", [0, 1])
def test_vcycle_parity_under_relaxed(qn, coupled):
    """omega_vanka = 0.8 (every block update scaled by omega on both sides):
    V-cycles from the level-n state, per-level and fused coarse levels."""
    P = W.small_case(32, 48, False)
    g = qn.Solver(**P.create_kwargs(), omega_vanka=0.8, coupled=coupled)
    r = RefSolver(**P.create_kwargs(), omega_vanka=0.8, coupled=coupled)
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        ng = g.vcycle()
        nr = r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-9 if coupled else 1e-10)
        assert np.allclose(ng, nr, rtol=1e-6, atol=1e-14)


def _step_both(qn, P, steps=1, **opt):
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **opt)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opt)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    hist = []
    for _ in range(steps):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        hist.append((ng, nr, resg, resr))
    return g, r, hist


@pytest.mark.parametrize("px", [False, True])
def test_full_step_parity_small(qn, px):
    P = W.small_case(32, 48, px)
    g, r, hist = _step_both(qn, P, steps=2)
    for ng, nr, resg, resr in hist:
        assert ng == nr and resg <= P.tol and resr <= P.tol
    fg, fr = g.get_fields(), r.get_fields()
    same_fields(fg, fr, 1e-10)
    mg, mr = g.mass(), r.mass()
    assert abs(mg[0] - mr[0]) <= 1e-13 * mr[0] and abs(mg[1] - mr[1]) <= 1e-13 * mr[1]
    eg, dg = g.energy()
    assert abs(eg - r.energy()) <= 1e-12 * abs(r.energy()) and dg > 0


def test_capillary_wave_64_parity(qn):
    P = W.capillary_64()
    P.steps = 3
    g, r, hist = _step_both(qn, P, steps=P.steps)
    same_fields(g.get_fields(), r.get_fields(), 1e-10)
    m0 = r.mass()


def test_rising_drop_full_size_one_step(qn):
    """The benchmark workload (256x512, 8 levels, tol 1e-9), one step, every field."""
    P = W.rising_drop_256x512()
    g, r, hist = _step_both(qn, P, steps=1)
    (ng, nr, resg, resr), = hist
    assert ng == nr
    same_fields(g.get_fields(), r.get_fields(), 1e-10)


def test_conservation_and_energy_on_gpu(qn):
    P = W.small_case(64, 64, False, rho_ratio=10.0)
    g = qn.Solver(**P.create_kwargs(), tol=1e-11)
    g.set_fields(P.fields())
    m0 = g.mass()
    e0, _ = g.energy()
    prev = e0
    for _ in range(3):
        g.step(P.dt)
        e, d = g.energy()
        assert e < prev and d > 0
        prev = e
    m1 = g.mass()
    assert abs(m1[0] - m0[0]) <= 1e-12 * m0[0]
    assert abs(m1[1] - m0[1]) <= 1e-12 * m0[1]


def test_device_field_io_roundtrip(qn):
    import torch
    P = W.small_case(24, 16, True)
    g = qn.Solver(**P.create_kwargs())
    f = W.random_state(24, 16, True, seed=3)
    t = {k: torch.tensor(v, device="cuda", dtype=torch.float64) for k, v in f.items()}
    g.set_fields_device(t)
    back = g.get_fields()
    for k in f:
        assert np.array_equal(back[k], f[k]), k
    out = {k: torch.empty_like(v) for k, v in t.items()}
    g.get_fields_device(out)
    for k in f:
        assert np.array_equal(out[k].cpu().numpy(), f[k]), k


def test_error_statuses(qn):
    with pytest.raises(qn.QnschError) as e:
        qn.Solver(7, 8, periodic_x=True)  # periodic x needs an even m1
    assert e.value.code == -1
    with pytest.raises(qn.QnschError):
        qn.Solver(16, 16, levels=9)
    g = qn.Solver(16, 16)
    with pytest.raises(qn.QnschError) as e:
        g.vcycle()  # no pending step
    assert e.value.code == -8
    with pytest.raises(qn.QnschError) as e:
        g.set_option("no_such_option", 1.0)
    assert e.value.code == -1
    P = W.small_case(16, 16, False)
    g = qn.Solver(**P.create_kwargs(), tol=1e-14, maxcyc=1)
    f = P.fields()
    g.set_fields(f)
    with pytest.raises(qn.QnschError) as e:
        g.step(P.dt)
    assert e.value.code == -4
    assert np.array_equal(g.get_fields()["c"], f["c"])  # not committed


# ---------------------------------------------------------------------------
# defect correction on the error equation (precision 2: FP64, 1: FP32 inner)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m1,m2,px", [(32, 48, False), (32, 48, True)])
def test_error_form_fp64_cycles_match_oracle(qn, m1, m2, px):
    """FAS on N(x+e) - N(x) = r(x) followed by x += e is the same algorithm as FAS
    on N(x) = 0 (the coarse problems differ only by the constant N_H(R x)), so in
    FP64 its iterates must match the oracle's direct V-cycles."""
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs(), precision=2)
    r = RefSolver(**P.create_kwargs())
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        ng = g.vcycle()
        nr = r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-9)
        assert np.allclose(ng, nr, rtol=1e-5, atol=1e-14)


@pytest.mark.parametrize("case", ["small_walls", "small_periodic", "drop_256x512"])
def test_mixed_precision_step_meets_fp64_tolerance(qn, case):
    """Precision 1: the FP64 residual meets tol, the fields agree with the FP64
    oracle's converged step, and mass is conserved to FP64 accuracy."""
    if case == "drop_256x512":
        P = W.rising_drop_256x512()
    else:
        P = W.small_case(32, 48, case.endswith("periodic"))
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    m0 = g.mass()
    ng, resg = g.step(P.dt)
    nr, resr = r.step(P.dt)
    assert resg <= P.tol and abs(ng - nr) <= 1
    check_mixed(g.get_fields(), r.get_fields())
    m1 = g.mass()
    assert abs(m1[0] - m0[0]) <= 1e-12 * m0[0] and abs(m1[1] - m0[1]) <= 1e-12 * m0[1]


@pytest.mark.parametrize("precision,px", [(0, False), (0, True), (1, False), (1, True)])
def test_fused_coarse_levels_match_per_level_launches(qn, precision, px):
    """The single-block V-cycle of the small levels (FP64: four-lane Vanka teams
    on the smallest) runs the same arithmetic in the same colour order as the
    per-level launches: the iterates agree to rounding."""
    P = W.small_case(64, 96, px)
    f = P.fields()
    out = []
    for fuse in (0, 10 ** 6):
        g = qn.Solver(**P.create_kwargs(), precision=precision, fuse_cells=fuse,
                      fuse_cells32=fuse)
        g.set_fields(f)
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[0], out[1], 1e-12 if precision == 0 else 1e-5)


# ---------------------------------------------------------------------------
# coupled 7x7 smoother (option)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m1,m2,px", [(16, 12, False), (16, 12, True), (37, 29, False)])
def test_coupled_sweep_parity(qn, m1, m2, px):
    g, r = pair(qn, m1, m2, px)
    g.set_option("coupled", 1)
    r.set_option("coupled", 1)
    load_random(g, r, px, seed=47)
    g.smooth(1)
    r.smooth(1)
    same_fields(g.get_iterate(), r.get_iterate(), 1e-10)


@pytest.mark.parametrize("precision", [0, 2])
def test_coupled_vcycle_parity(qn, precision):
    P = W.small_case(64, 96, False)
    g = qn.Solver(**P.create_kwargs(), coupled=1, precision=precision)
    r = RefSolver(**P.create_kwargs(), coupled=1)
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        g.vcycle()
        r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-9)


def test_coupled_full_step_rising_drop(qn):
    P = W.rising_drop_256x512()
    g, r, hist = _step_both(qn, P, steps=1, coupled=1)
    (ng, nr, resg, resr), = hist
    assert ng == nr and resg <= P.tol
    same_fields(g.get_fields(), r.get_fields(), 1e-10)


def test_coupled_mixed_step_512(qn):
    """Fine grid where the separate sweeps stall: the coupled block converges in
    both the FP64 oracle and the mixed GPU path, to the same fields."""
    P = W.rising_drop_256x512()
    P.m1, P.m2 = 512, 512
    P.init_args = dict(x0=0.5, y0=0.3, R=0.2)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, coupled=1, precision=1)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, coupled=1)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    ng, resg = g.step(P.dt)
    nr, resr = r.step(P.dt)
    assert resg <= P.tol and abs(ng - nr) <= 1
    check_mixed(g.get_fields(), r.get_fields())


def _rt(m1, m2):
    P = W.rayleigh_taylor_1024x4096()
    P.m1, P.m2 = m1, m2
    P.Cn = 2.5 / m1
    P.Pe = 1.0 / P.Cn
    return P


@pytest.mark.parametrize("coupled,fuse", [(0, 512), (1, 512), (0, 0)])
def test_vcycle_parity_tall_periodic(qn, coupled, fuse):
    """Periodic 1 x 4 box: width stops at 4, coarsest grid 4 x 16 with the
    scaled coarsest sweeps; fused and per-level coarse paths both match."""
    P = _rt(64, 256)
    g = qn.Solver(**P.create_kwargs(), coupled=coupled, fuse_cells=fuse)
    r = RefSolver(**P.create_kwargs(), coupled=coupled)
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    assert g.levels == r.levels == 5
    for _ in range(3):
        ng = g.vcycle()
        nr = r.vcycle()
        same_fields(g.get_iterate(), r.get_iterate(), 1e-10)
        assert np.allclose(ng, nr, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("precision,coupled", [(0, 1), (1, 1), (1, 0)])
def test_rayleigh_taylor_full_size_step(qn, precision, coupled):
    """Rayleigh-Taylor 1024 x 4096 (4.2 M cells, 9 levels): one step converges
    (the mixed paper smoother runs one lane per Vanka block on the finest
    level, four on the others); the oracle's own residual of the GPU's new
    state is at the tolerance, and mass is conserved to round-off."""
    P = W.rayleigh_taylor_1024x4096()
    f0 = P.fields()
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, coupled=coupled, precision=precision)
    g.set_fields(f0)
    m0 = g.mass()
    ng, res = g.step(P.dt)
    assert res <= P.tol and ng < 50
    f1 = g.get_fields()
    m1 = g.mass()
    assert abs(m1[0] - m0[0]) <= 1e-12 * abs(m0[0]) and abs(m1[1] - m0[1]) <= 1e-12 * abs(m0[1])
    r = RefSolver(**P.create_kwargs(), tol=P.tol, coupled=coupled)
    r.set_fields(f0)
    r.begin_step(P.dt)
    r.set_iterate(f1)
    _, norms = r.residual()
    assert max(norms[:5]) <= 2 * P.tol, norms[:5]


@pytest.mark.parametrize("px", [False, True])
@pytest.mark.parametrize("coupled", [0, 1])
def test_team_vanka_launches_match_single_lane(qn, px, coupled):
    """Per-level Vanka (or coupled-block) and CH launches with four lanes per
    block (vanka_team_max, ch_team_max) do the same arithmetic as one lane per
    block, with some terms summed in another order: after two V-cycles the
    iterates agree within the 1e-10 parity bar (measured 2e-12)."""
    P = W.small_case(128, 192, px)
    out = []
    for tm in (0, 10 ** 9):
        g = qn.Solver(**P.create_kwargs(), vanka_team_max=tm, ch_team_max=tm, coupled=coupled,
                      fuse_cells=0)
        g.set_fields(P.fields())
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[0], out[1], 1e-10)


@pytest.mark.parametrize("coupled", [0, 1])
@pytest.mark.parametrize("precision,tol", [(2, 1e-10), (1, 1e-5)])
def test_team_vanka_on_error_levels_matches_single_lane(qn, precision, tol, coupled):
    """The error-equation levels of the defect correction (FP64 check form and
    FP32) smoothed with four lanes per Vanka (or coupled) block and per CH cell
    agree with one lane per block: to the parity bar in FP64, to FP32 rounding
    in the mixed cycle."""
    P = W.small_case(128, 192, False)
    out = []
    for tm in (0, 10 ** 9):
        g = qn.Solver(**P.create_kwargs(), precision=precision, vanka_team_max32=tm,
                      ch_team_max32=tm, fuse_cells32=0, coupled=coupled)
        g.set_fields(P.fields())
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[0], out[1], tol)
