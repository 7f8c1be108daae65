"""Sec. 9 self-convergence study on the GPU: levels 16 and 32 equal the
oracle's, and the Cauchy differences of c up to m = 256 fall at second order."""
import numpy as np
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import convergence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    from paper_1703_06606_gb300 import qnsch
    return qnsch


@pytest.mark.parametrize("m", [16, 32])
def test_convergence_levels_match_oracle(qn, m):
    fg, ig = convergence.solve(qn.Solver, m)
    fr, ir = convergence.solve(RefSolver, m)
    assert ig["vcycles_per_step"] == ir["vcycles_per_step"]
    for k in fr:
        scale = max(np.max(np.abs(fr[k])), 1e-30)
        assert np.max(np.abs(fg[k] - fr[k])) <= 1e-10 * scale, k


def test_self_convergence_second_order_to_256(qn):
    rows = convergence.run(qn.Solver, (16, 32, 64, 128, 256))
    e = [r["error"] for r in rows[1:]]
    assert all(e[k + 1] < e[k] for k in range(len(e) - 1)), rows
    assert 1.8 <= rows[-1]["rate"] <= 2.5 and 1.8 <= rows[-2]["rate"] <= 2.5, rows


def test_projection_self_convergence_second_order(qn):
    """The projection method on the same schedule from m = 32 (at m = 16,
    dt = 1/16 its point smoothers diverge): second-order Cauchy rates, as in
    the projection column of the paper's Table 1."""
    rows = convergence.run(qn.Solver, (32, 64, 128, 256), scheme=1)
    e = [r["error"] for r in rows[1:]]
    assert all(e[k + 1] < e[k] for k in range(len(e) - 1)), rows
    assert 1.7 <= rows[-1]["rate"] <= 2.5, rows
