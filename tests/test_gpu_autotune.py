"""The autotuner on the GPU: tuning a small case measures real steps, and the
tuned options leave the step's result where the defaults put it."""
import numpy as np
import pytest

from paper_1703_06606_gb300 import autotune
from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qn():
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def test_tuned_options_keep_the_step(qn):
    P = W.capillary_64()
    # launch shapes only: the smoothing counts stay at their defaults here, so
    # the tuned step must take the defaults' V-cycles (other counts change the
    # iteration, not the answer)
    cand = {"vanka_team_max32": [131072, 0], "ch_team_max32": [0, 4096],
            "fuse_cells32": [512, 2048], "wave_cells32": [0, 1024], "wave_rows": [8, 4],
            "skew_cells32": [0, 1024], "skew_rows": [32, 4], "nu1": [2], "nu2": [2],
            "nu_coarse": [4], "nu1_fine": [-1], "nu2_fine": [-1]}
    best, t, hist = autotune.tune(P, precision=1, coupled=1, steps=2, warmup=1, candidates=cand)
    assert t is not None and t > 0 and len(hist) >= 4
    assert set(best) == set(autotune.KNOBS[1])
    out = []
    for opts in ({}, best):
        s = qn.Solver(**P.create_kwargs(), tol=P.tol, precision=1, coupled=1, **opts)
        s.set_fields(P.fields())
        n = [s.step(P.dt)[0] for _ in range(3)]
        out.append((n, s.get_fields()))
        s.close()
    assert out[0][0] == out[1][0]
    # two mixed-precision paths, each within the mixed bar of the FP64 solution
    from mixed_tol import MIXED_TOL
    for k in out[0][1]:
        a, b = out[0][1][k], out[1][1][k]
        assert np.max(np.abs(a - b)) <= 2 * MIXED_TOL[k] * max(np.max(np.abs(a)), 1e-30), k


def test_server_applies_the_table(qn):
    from paper_1703_06606_gb300 import serve
    P = W.capillary_64()
    dev = autotune.device_name()
    table = {autotune.key_of(P, 1, 1, 0, dev): {"options": {"fuse_cells32": 2048}, "ms_per_step": 1.0}}
    srv = serve.Server(tuned_table=table)
    assert srv.options(P) == {"fuse_cells32": 2048}
    other = W.small_case(32, 48, False)
    assert srv.options(other) == {}
