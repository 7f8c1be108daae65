"""The self-convergence study of Sec. 9 (Table 1) in the oracle: the bilinear
push-up is exact for linear fields and keeps constants; with dt = 16 h^2 the
Cauchy differences of c fall at second order."""
import numpy as np

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import convergence


def test_bilinear_push_up_is_exact_for_linear_fields():
    m1, m2 = 12, 10
    h = 1.0 / m1
    x = (np.arange(1, m1 + 1) - 0.5) * h
    y = (np.arange(1, m2 + 1) - 0.5) * h
    a = 1.0 + 2.0 * x[None, :] - 3.0 * y[:, None]
    f = convergence.prolong_bilinear(a)
    xf = (np.arange(1, 2 * m1 + 1) - 0.5) * h / 2
    yf = (np.arange(1, 2 * m2 + 1) - 0.5) * h / 2
    want = 1.0 + 2.0 * xf[None, :] - 3.0 * yf[:, None]
    assert np.max(np.abs(f[1:-1, 1:-1] - want[1:-1, 1:-1])) <= 1e-14
    assert np.max(np.abs(convergence.prolong_bilinear(np.full((m2, m1), 0.7)) - 0.7)) <= 1e-15


def test_oracle_self_convergence_is_second_order():
    rows = convergence.run(RefSolver, (16, 32, 64))
    e = [r["error"] for r in rows[1:]]
    assert e[1] < e[0] / 3.0 and rows[2]["rate"] >= 1.8, rows


def test_oracle_projection_self_convergence_is_second_order():
    """The projection method (Sec. 6.2) on the Sec. 9 schedule from m = 32:
    the Cauchy difference falls at second order (rate 1.95 at 64 & 128)."""
    rows = convergence.run(RefSolver, (32, 64, 128), scheme=1)
    e = [r["error"] for r in rows[1:]]
    assert e[1] < e[0] / 3.0 and rows[2]["rate"] >= 1.8, rows
