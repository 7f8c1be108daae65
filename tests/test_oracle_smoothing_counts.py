"""Smoothing counts in the oracle's V-cycle (options nu1, nu2 on every level,
nu1_fine, nu2_fine on the finest level only).  The counts change the
iteration, not the discrete solution: with the finest level's counts equal to
the others' (or -1) the steps are bit for bit those of the defaults; with
counts of its own the step still converges to the same tolerance and to the
same state within what that tolerance allows, by a different iteration; the
options read back."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W


def _run(P, steps=3, **opts):
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    r.set_fields(P.fields())
    cyc = [r.step(P.dt)[0] for _ in range(steps)]
    return cyc, r.get_fields()


def test_equal_fine_counts_are_the_defaults():
    P = W.small_case(32, 32, True)
    base = _run(P)
    for opts in ({"nu1_fine": -1, "nu2_fine": -1}, {"nu1_fine": 2, "nu2_fine": 2}):
        got = _run(P, **opts)
        assert got[0] == base[0]
        assert all(np.array_equal(got[1][k], base[1][k]) for k in base[1])


@pytest.mark.parametrize("fine,coarse", [((3, 2), (1, 1)), ((2, 3), (1, 1)), ((1, 2), (2, 2))])
def test_own_fine_counts_reach_the_same_state(fine, coarse):
    P = W.small_case(32, 48, False)
    base_cyc, base = _run(P, steps=4)
    cyc, f = _run(P, steps=4, nu1=coarse[0], nu2=coarse[1], nu1_fine=fine[0], nu2_fine=fine[1])
    for k in f:
        e = np.max(np.abs(f[k] - base[k])) / max(np.max(np.abs(base[k])), 1e-300)
        assert e <= 1e-6, (k, e)


def test_the_fine_counts_take_effect():
    """Other counts on the finest level change the iteration (not the
    answer): the V-cycle counts or the last bits of the state differ."""
    P = W.small_case(32, 48, False)
    base_cyc, base = _run(P, steps=2)
    cyc, f = _run(P, steps=2, nu1_fine=3, nu2_fine=2)
    assert cyc != base_cyc or any(not np.array_equal(f[k], base[k]) for k in f)


def test_fine_options_read_back():
    P = W.small_case(16, 16, False)
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    assert r.get_option("nu1_fine") == -1 and r.get_option("nu2_fine") == -1
    r.set_option("nu1_fine", 3)
    r.set_option("nu2_fine", 0)
    assert r.get_option("nu1_fine") == 3 and r.get_option("nu2_fine") == 0
