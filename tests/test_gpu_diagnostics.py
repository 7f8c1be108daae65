"""GPU diagnostics of Sec. 8 (qnsch_diagnostics, qnsch_divergence) against the
oracle on the same states: closed-form states, states after GPU and oracle
steps, and the full-size workloads."""
import math

import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def _both(qn, P, fields, **opt):
    g = qn.Solver(**P.create_kwargs(), **opt)
    r = RefSolver(**P.create_kwargs(), **opt)
    g.set_fields(fields)
    r.set_fields(fields)
    return g, r


def _close(dg, dr, rtol, floor=1e-12, fields=None, h=None):
    """|gpu - oracle| <= rtol * max(|oracle|, floor) for every diagnostic; with
    `fields`, V_c is measured on the velocity scale max|v| and the divergence
    terms on max|v| / h (a divergence at the solver tolerance is noise)."""
    for k in dr:
        scale = max(abs(dr[k]), floor)
        if fields is not None and k == "Vc":
            scale = max(scale, np.max(np.abs(fields["v"])))
        if fields is not None and k.startswith("div"):
            scale = max(scale, np.max(np.abs(fields["v"])) / h)
        assert abs(dg[k] - dr[k]) <= rtol * scale, (k, dg[k], dr[k])


@pytest.mark.parametrize("m1,m2,px", [(32, 16, True), (37, 29, False), (300, 70, False)])
def test_diagnostics_of_random_state_match_oracle(qn, m1, m2, px):
    """Seeded random state (several tiles, ragged tails): every diagnostic and
    the divergence field agree with the oracle to rounding."""
    P = W.small_case(m1, m2, px)
    f = W.random_state(m1, m2, px, seed=11)
    g, r = _both(qn, P, f)
    dg, dr = g.diagnostics(), r.diagnostics()
    _close(dg, dr, 1e-12)
    vg, vr = g.divergence(), r.divergence()
    assert np.max(np.abs(vg - vr)) <= 1e-12 * np.max(np.abs(vr))


def test_diagnostics_of_interface_states_match_oracle(qn):
    """Piecewise-linear RT interface (exact tips) and the tanh capillary wave."""
    P = W.rayleigh_taylor_1024x4096()
    P.m1, P.m2 = 64, 256
    x = (np.arange(1, 65) - 0.5) / 64
    yt = 2.0 + 0.1 * np.cos(2 * math.pi * x)
    y = (np.arange(1, 257) - 0.5) / 64
    f = P.fields()
    f["c"] = np.clip(0.5 - (y[:, None] - yt[None, :]) * 16.0, 0.0, 1.0)
    g, r = _both(qn, P, f)
    dg = g.diagnostics()
    assert abs(dg["y_top"] - yt.max()) <= 1e-12 and abs(dg["y_bottom"] - yt.min()) <= 1e-12
    _close(dg, r.diagnostics(), 1e-12)
    C = W.capillary_64()
    C.m1 = C.m2 = 128
    g, r = _both(qn, C, C.fields())
    dg = g.diagnostics()
    assert abs(dg["a1"] - 0.01) <= 1e-12
    _close(dg, r.diagnostics(), 1e-12)


@pytest.mark.parametrize("case", ["capillary_64", "small_walls"])
def test_diagnostics_after_steps_match_oracle(qn, case):
    P = W.capillary_64() if case == "capillary_64" else W.small_case(48, 64, False, rho_ratio=10.0)
    steps = 3
    g = qn.Solver(**P.create_kwargs(), tol=P.tol)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    for _ in range(steps):
        g.step(P.dt)
        r.step(P.dt)
    dg, dr = g.diagnostics(), r.diagnostics()
    # the fields agree to 1e-10 relative, so the diagnostics to 1e-8 of their scale
    fr = r.get_fields()
    _close(dg, dr, 1e-8, fields=fr, h=g.h)
    vr = r.divergence()
    assert np.max(np.abs(g.divergence() - vr)) <= 1e-8 * np.max(np.abs(fr["v"])) / g.h


def test_rising_drop_full_size_diagnostics(qn):
    """Bench workload after one step: every diagnostic equals the oracle's."""
    P = W.rising_drop_256x512()
    g = qn.Solver(**P.create_kwargs(), tol=P.tol)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    g.step(P.dt)
    r.step(P.dt)
    dg, dr = g.diagnostics(), r.diagnostics()
    _close(dg, dr, 1e-8, fields=r.get_fields(), h=g.h)


def test_light_drop_rises(qn):
    """After the first steps' interface relaxation (V_c briefly < 0), the light
    drop rises: V_c > 0 and growing, the centroid moves up; GPU = oracle."""
    P = W.rising_drop_256x512()
    P.m1, P.m2, P.Cn, P.Pe = 64, 128, 0.02, 50.0
    g = qn.Solver(**P.create_kwargs(), tol=1e-9)
    r = RefSolver(**P.create_kwargs(), tol=1e-9)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    y0 = g.diagnostics()["yc"]
    hist = []
    for _ in range(12):
        g.step(1e-3)
        r.step(1e-3)
        hist.append(g.diagnostics()["Vc"])
    d = g.diagnostics()
    assert hist[-1] > hist[-4] > 0 and d["yc"] > y0
    _close(d, r.diagnostics(), 1e-8, fields=r.get_fields(), h=g.h)


def test_rayleigh_taylor_full_size_initial_diagnostics(qn):
    """1024 x 4096 initial state: every diagnostic equals the oracle's."""
    P = W.rayleigh_taylor_1024x4096()
    f = P.fields()
    g, r = _both(qn, P, f)
    dg, dr = g.diagnostics(), r.diagnostics()
    _close(dg, dr, 1e-12)
    assert abs(dg["y_top"] - 2.1) < 1e-3 and abs(dg["y_bottom"] - 1.9) < 1e-3
