"""Pins of the oracle's projection method (Sec. 6.2, solver Sec. 7.2) against
what the paper and the mathematics fix:
  * the discrete energy identity behind the projection method's energy
    theorem, for arbitrary states (every term of every family, and the
    placement of gravity in the projection equation);
  * the pointwise continuity identity behind its mass theorem, and exact
    conservation of sum(rho) and sum(rho c) after converged steps;
  * Newton with a direct solve on tiny grids against the multigrid fixed point;
  * rho1 = rho2: the projected velocity is discretely divergence free."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W

from test_oracle_pins import _newton, make, rho_fn, u_cols


def _random_pending(px, seed, dt=2e-3):
    s = make(16, 12, px, scheme=1)
    fn = W.random_state(16, 12, px, seed=seed)
    s.set_fields(fn)
    s.begin_step(dt)
    s.set_iterate(W.random_state(16, 12, px, seed=seed + 100))
    return s, fn, dt


@pytest.mark.parametrize("px", [False, True])
@pytest.mark.parametrize("seed", [1, 2])
def test_projection_energy_identity_arbitrary_state(px, seed):
    """h^2 [dt(ut, N_ut) + dt(vt, N_vt) + dt/M (mu, N_c) + dt/M (p, N_p)
    - 1/M (c - c^n, N_mu) + dt/Fr (y, -alpha rho(c) N_c + rho(c) N_p)]
    = E(c, u^{n+1}) - E^n + D, with D the viscous and CH dissipation of the
    intermediate velocity, 1/2||sqrt(rho^n)(ut - u^n)||^2 and
    1/2||sqrt(rho(c))(u^{n+1} - ut)||^2: the test functions of the projection
    method's energy proof make every term telescope.  Gravity must act in the
    projection equation for this to hold (with A rho^{n+1} in the
    intermediate-velocity row, as printed, it fails by ~2e-5 relative)."""
    s, fn, dt = _random_pending(px, seed)
    x = s.get_iterate()
    r, _ = s.residual()
    N = {k: -v for k, v in r.items()}
    P = s.params()
    h, M, alpha, Fr_inv = P["h"], P["M"], P["alpha"], P["Fr_inv"]
    rho = rho_fn(x["c"], 1.0, 3.0)
    y = ((np.arange(1, 13) - 0.5) * h)[:, None]
    cols = u_cols(s)
    terms = [dt * np.sum(x["u"][:, cols] * N["u"][:, cols]),
             dt * np.sum(x["v"][1:-1, :] * N["v"][1:-1, :]),
             dt / M * np.sum(x["mu"] * N["c"]),
             dt / M * np.sum(x["p"] * N["p"]),
             -1.0 / M * np.sum((x["c"] - fn["c"]) * N["mu"]),
             dt * Fr_inv * np.sum(y * (-alpha * rho * N["c"] + rho * N["p"]))]
    lhs = h * h * sum(terms)
    rhs = s.iterate_energy() - s.energy() + s.iterate_dissipation()
    scale = h * h * sum(abs(t) for t in terms)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs, scale)
    # a planted sign error in one family breaks it
    bad = lhs - 2 * h * h * terms[4]
    assert abs(bad - rhs) > 1e-3 * abs(rhs)


@pytest.mark.parametrize("px", [False, True])
def test_projection_pointwise_continuity(px):
    """-alpha rho(c) N_c + rho(c) N_p = (rho(c) - rho^n)/dt + d_x(A_x rho(c) u^{n+1})
    + d_y(A_y rho(c) v^{n+1}) cell by cell, for any state (the secant identity
    rho_a - rho_b = -alpha rho_a rho_b (c_a - c_b) turns the advection of
    (pj-num-phase) into a flux difference)."""
    s, fn, dt = _random_pending(px, 3)
    x = s.get_iterate()
    r, _ = s.residual()
    P = s.params()
    h, alpha = P["h"], P["alpha"]
    u, v = s.projected_velocity()
    rho = rho_fn(x["c"], 1.0, 3.0)
    rhon = rho_fn(fn["c"], 1.0, 3.0)
    m2, m1 = rho.shape
    # face densities A_x rho(c) on the m1+1 x-edges (periodic wrap or wall copy)
    rpad = np.concatenate([rho[:, -1:], rho, rho[:, :1]], axis=1) if px else \
        np.concatenate([rho[:, :1], rho, rho[:, -1:]], axis=1)
    Axr = 0.5 * (rpad[:, :-1] + rpad[:, 1:])
    Ayr = np.zeros((m2 + 1, m1))
    Ayr[1:-1, :] = 0.5 * (rho[:-1, :] + rho[1:, :])
    fx = Axr * u
    fy = Ayr * v
    div = (fx[:, 1:] - fx[:, :-1]) / h + (fy[1:, :] - fy[:-1, :]) / h
    lhs = -alpha * rho * (-r["c"]) + rho * (-r["p"])
    rhs = (rho - rhon) / dt + div
    assert np.max(np.abs(lhs - rhs)) <= 1e-11 * np.max(np.abs(rhs))


@pytest.mark.parametrize("px", [False, True])
def test_projection_mass_conserved_after_steps(px):
    P = W.small_case(32, 48, px, rho_ratio=10.0)
    s = RefSolver(**P.create_kwargs(), tol=1e-12, maxcyc=60, scheme=1)
    s.set_fields(P.fields())
    m0 = s.mass()
    E = [s.energy()]
    for _ in range(3):
        n, res = s.step(P.dt)
        assert res <= 1e-12
        E.append(s.energy())
    m1 = s.mass()
    assert abs(m1[0] - m0[0]) <= 1e-13 * m0[0] and abs(m1[1] - m0[1]) <= 1e-13 * m0[1]
    assert all(E[k + 1] < E[k] for k in range(3)), E


@pytest.mark.parametrize("m1,m2,px", [(8, 8, False), (8, 8, True), (8, 12, False)])
def test_projection_fixed_point_equals_newton_direct_solve(m1, m2, px):
    P = W.small_case(m1, m2, px)
    P.Cn, P.Pe = 0.1, 10.0
    s = RefSolver(**P.create_kwargs(), tol=1e-13, maxcyc=200, scheme=1)
    f0 = P.fields()
    s.set_fields(f0)
    s.begin_step(P.dt)
    while max(s.vcycle()[:5]) > 1e-13:
        pass
    xm = s.get_iterate()
    s.set_iterate({k: f0[k] for k in f0})
    xn, fres = _newton(s, s.get_iterate())
    assert fres < 1e-11
    xn["p"] -= xn["p"].mean()
    for k in xm:
        scale = max(np.max(np.abs(xm[k])), 1e-8)
        assert np.max(np.abs(xm[k] - xn[k])) <= 1e-10 * max(scale, 1.0), k


def test_projection_equal_densities_divergence_free():
    """rho1 = rho2 (alpha = 0): (pj-num-mass) reads d.u^{n+1} = 0."""
    P = W.small_case(32, 32, True, rho_ratio=1.0)
    s = RefSolver(**P.create_kwargs(), tol=1e-12, maxcyc=60, scheme=1)
    s.set_fields(P.fields())
    s.step(P.dt)
    s.begin_step(P.dt)
    while max(s.vcycle()[:5]) > 1e-12:
        pass
    u, v = s.projected_velocity()
    div = (u[:, 1:] - u[:, :-1]) * 32 + (v[1:, :] - v[:-1, :]) * 32
    assert np.max(np.abs(div)) <= 1e-9


def test_projection_vcycle_contracts():
    for P in (W.small_case(32, 32, True), W.small_case(32, 48, False)):
        s = RefSolver(**P.create_kwargs(), scheme=1)
        s.set_fields(P.fields())
        s.begin_step(P.dt)
        hist = [max(s.vcycle()[:5]) for _ in range(6)]
        rates = [hist[k + 1] / hist[k] for k in range(1, 5)]
        assert max(rates) < 0.2, hist


def test_projection_option_rules():
    s = RefSolver(16, 16, scheme=1)
    with pytest.raises(Exception):
        s.set_option("coupled", 1)
    t = RefSolver(16, 16, coupled=1)
    with pytest.raises(Exception):
        t.set_option("scheme", 1)
