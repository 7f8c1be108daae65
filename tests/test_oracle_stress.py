"""The high-ratio stress cases (capillary wave at density ratio 1:1000 and the
paper's own droplet parameters, Sec. 8.1-8.2) at reduced size in the oracle:
every step converges with both smoothers, Thm. 6.1's masses are conserved and
Thm. 6.2's energy does not increase."""
import pytest

from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W


def _reduced(name):
    P = getattr(W, name)()
    scale = P.m1 // 32
    P.m1, P.m2 = P.m1 // scale, P.m2 // scale
    P.Cn *= scale
    P.Pe = 1.0 / P.Cn
    return P


@pytest.mark.parametrize("name", ["capillary_ratio1000_256", "droplet_paper_256x512"])
@pytest.mark.parametrize("coupled", [0, 1])
def test_stress_case_converges_conserves_and_dissipates(name, coupled):
    P = _reduced(name)
    s = RefSolver(**P.create_kwargs(), tol=P.tol, maxcyc=40, coupled=coupled)
    s.set_fields(P.fields())
    m0 = s.mass()
    E = [s.energy()]
    for _ in range(4):
        n, res = s.step(P.dt)
        assert res <= P.tol and n < 40
        E.append(s.energy())
    m1 = s.mass()
    assert abs(m1[0] - m0[0]) <= 1e-12 * m0[0] and abs(m1[1] - m0[1]) <= 1e-12 * m0[1]
    assert all(E[k + 1] <= E[k] + 1e-12 * abs(E[k]) for k in range(4)), E
