"""The oracle's predicted initial iterate (option "predictor"): the step starts
from the polynomial in time through the committed state and the one or two
states committed before it, evaluated at the new time.  Pinned by what an
extrapolation on unequal nodes must do: degree 2 reproduces any state that is
quadratic in time exactly and degree 1 any linear one, degree 1 misses a
quadratic by exactly C dt (dt + a), and with fewer states held the degree
drops.  Also the bookkeeping (history kept by committed steps only, not
counting the state the caller set, cleared by set_fields and by setting the
option, set/get round trip) and that the
predictor changes where the outer cycles start, not the answer: the step
converges to the same residual tolerance with fewer V-cycles once the
history is full."""
import numpy as np
import pytest

from oracle.ref import RefError, RefSolver
from paper_1703_06606_gb300 import workloads as W


def _states(P, seed):
    """Three seeded random states that satisfy the boundary conditions once set."""
    out = []
    for k in range(3):
        f = W.random_state(P.m1, P.m2, P.periodic_x, seed=seed + k)
        out.append(f)
    return out


def _quadratic(S, t):
    """F(t) = A + B t + C t^2 from the three states A, B, C."""
    A, B, C = S
    return {k: A[k] + t * B[k] + t * t * C[k] for k in A}


def _bc(r, f):
    """f with the boundary values the solver gives it (round trip through set_fields)."""
    r.set_fields(f)
    return r.get_fields()


def _predicted(P, order, fields_t, dt, hist):
    """The oracle's initial iterate of a step of size dt from fields_t with
    history hist = [(fields, dt), ...] (most recent first)."""
    r = RefSolver(**P.create_kwargs(), tol=P.tol, predictor=order)
    r.set_fields(fields_t)
    for k, (f, h) in enumerate(hist):
        r.set_history(k, f, h)
    r.begin_step(dt)
    x0 = r.get_iterate()
    r.close()
    return x0


@pytest.mark.parametrize("periodic", [False, True])
def test_degree_two_reproduces_a_quadratic_in_time_on_unequal_steps(periodic):
    P = W.small_case(12, 16, periodic)
    ref = RefSolver(**P.create_kwargs(), tol=P.tol)
    S = [_bc(ref, f) for f in _states(P, 11)]
    a, b, dt = 0.7e-3, 1.3e-3, 0.9e-3  # the last two steps and the next one
    t0 = 0.37
    F = lambda t: _quadratic(S, t)  # noqa: E731
    x0 = _predicted(P, 2, F(t0), dt, [(F(t0 - a), a), (F(t0 - a - b), b)])
    want = F(t0 + dt)
    for k in want:
        assert np.max(np.abs(x0[k] - want[k])) <= 1e-12 * max(np.max(np.abs(want[k])), 1.0), k


def test_degree_one_reproduces_a_line_and_misses_a_quadratic_by_its_error_term():
    P = W.small_case(12, 16, False)
    ref = RefSolver(**P.create_kwargs(), tol=P.tol)
    A, B, C = [_bc(ref, f) for f in _states(P, 21)]
    a, dt, t0 = 1.1e-3, 0.6e-3, 0.5
    line = lambda t: {k: A[k] + t * B[k] for k in A}  # noqa: E731
    x0 = _predicted(P, 1, line(t0), dt, [(line(t0 - a), a)])
    for k in A:
        assert np.max(np.abs(x0[k] - line(t0 + dt)[k])) <= 1e-12 * max(np.max(np.abs(A[k])), 1.0)
    quad = lambda t: {k: A[k] + t * B[k] + t * t * C[k] for k in A}  # noqa: E731
    x0 = _predicted(P, 1, quad(t0), dt, [(quad(t0 - a), a)])
    # linear extrapolation of t^2 from t0 - a, t0 to t0 + dt misses by dt (dt + a)
    for k in A:
        err = quad(t0 + dt)[k] - x0[k]
        assert np.allclose(err, dt * (dt + a) * C[k], rtol=1e-6, atol=1e-12), k


def test_the_degree_drops_to_what_the_history_holds():
    P = W.small_case(12, 16, True)
    ref = RefSolver(**P.create_kwargs(), tol=P.tol)
    A, B, _ = [_bc(ref, f) for f in _states(P, 31)]
    a, dt = 1e-3, 1e-3
    line = lambda t: {k: A[k] + t * B[k] for k in A}  # noqa: E731
    # order 2 with one earlier state: the line through the two states
    x0 = _predicted(P, 2, line(0.0), dt, [(line(-a), a)])
    for k in A:
        assert np.allclose(x0[k], line(dt)[k], rtol=1e-12, atol=1e-14), k
    # no earlier state, or order 0: the committed state itself
    for order, hist in ((2, []), (0, [(line(-a), a)])):
        x0 = _predicted(P, order, line(0.0), dt, hist)
        for k in A:
            assert np.array_equal(x0[k], line(0.0)[k]), (order, k)


def test_history_bookkeeping():
    P = W.small_case(16, 16, False)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, predictor=2)
    r.set_fields(P.fields())
    assert r.get_option("history") == 0
    states = [r.get_fields()]
    # the state set by the caller is no node (its mu and p are guesses), so
    # the history grows from the second committed step on
    for n in range(4):
        r.step(P.dt * (1.0 + 0.25 * n))
        states.append(r.get_fields())
        assert r.get_option("history") == min(n, 2)
    states = states[1:]
    h0, d0 = r.history(0)
    h1, d1 = r.history(1)
    assert d0 == P.dt * 1.75 and d1 == P.dt * 1.5
    for k in h0:
        assert np.array_equal(h0[k], states[2][k]) and np.array_equal(h1[k], states[1][k])
    with pytest.raises(RefError):
        r.history(2)
    # an uncommitted step leaves the history alone
    r.set_option("maxcyc", 1)
    r.set_option("tol", 1e-30)
    with pytest.raises(RefError):
        r.step(P.dt)
    assert r.get_option("history") == 2
    assert np.array_equal(r.history(0)[0]["c"], states[2]["c"])
    r.set_option("maxcyc", 50)  # a converged step ends the pending one
    r.set_option("tol", P.tol)
    r.step(P.dt)
    # set_fields and the option clear it; history 0 clears it
    r.set_fields(states[0])
    assert r.get_option("history") == 0
    r.set_history(0, states[1], P.dt)
    r.set_history(1, states[2], P.dt)
    assert r.get_option("history") == 2
    r.set_option("predictor", 1)
    assert r.get_option("history") == 0
    r.set_history(0, states[1], P.dt)
    r.set_option("history", 0)
    assert r.get_option("history") == 0
    with pytest.raises(RefError):
        r.set_history(1, states[1], P.dt)  # no gap
    with pytest.raises(RefError):
        r.set_option("history", 1)


def test_same_tolerance_fewer_cycles():
    """The capillary wave over ten steps: with either predictor every step
    reaches tol; the states stay within what the tolerance allows of the
    plain run's, and once the history is full the steps take fewer V-cycles."""
    P = W.capillary_64()
    runs = {}
    for order in (0, 1, 2):
        r = RefSolver(**P.create_kwargs(), tol=P.tol, predictor=order)
        r.set_fields(P.fields())
        cyc = []
        for _ in range(10):
            n, res = r.step(P.dt)
            assert res <= P.tol
            cyc.append(n)
        runs[order] = (cyc, r.get_fields())
    base = runs[0]
    for order in (1, 2):
        cyc, f = runs[order]
        assert sum(cyc[3:]) < sum(base[0][3:]), (order, cyc, base[0])
        for k in f:
            e = np.max(np.abs(f[k] - base[1][k])) / max(np.max(np.abs(base[1][k])), 1e-300)
            assert e <= 1e-6, (order, k, e)
