"""Mixed precision against the FP64 oracle, field by field, at the bars of
tests/mixed_tol.py (about ten times the measured differences), with V-cycle
counts within one of the oracle's and mass conserved: small cases with either
smoother, the option set of the batch and the server (serve.THROUGHPUT_OPTIONS:
coupled block, one lane per block in the per-level launches, levels up to
2048 cells fused, one smoothing step before the coarse-grid correction and two
after, each step from the quadratic extrapolation of the last three states,
the oracle running the same counts and predictor; four steps) on two draws of the
64-drop batch workload at density ratios 83 and 57, the 256x512 rising drop
with the per-colour smoother launches and with the banded wavefront, and a
512^2 drop with the coupled block.  Also the FP64 path at full size over
several steps: three steps of the 256x512 drop from the state the GPU reaches
after five, against the oracle from that same state."""
import numpy as np
import pytest

from mixed_tol import MIXED_MASS_TOL, check_mixed
from oracle.ref import RefSolver
from paper_1703_06606_gb300 import workloads as W
from paper_1703_06606_gb300.serve import THROUGHPUT_OPTIONS

pytestmark = pytest.mark.gpu

BATCH_OPTS = dict(precision=1, coupled=1, **THROUGHPUT_OPTIONS)
# the oracle follows the same algorithm: the coupled block, the smoothing
# counts and the predicted initial iterate
BATCH_REF = {"coupled": 1, **{k: THROUGHPUT_OPTIONS[k] for k in ("nu1", "nu2", "predictor")}}


@pytest.fixture(scope="module")
def qn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return qnsch


def _drop512():
    P = W.rising_drop_256x512()
    P.m1, P.m2 = 512, 512
    P.init_args = dict(x0=0.5, y0=0.3, R=0.2)
    return P


def _cases():
    ds = W.batch_drops(n=64)
    return [
        ("small_walls", W.small_case(32, 48, False), 1, {"precision": 1}, {}),
        ("small_periodic", W.small_case(32, 48, True), 1, {"precision": 1}, {}),
        ("small_walls_coupled", W.small_case(32, 48, False), 2, {"precision": 1, "coupled": 1},
         {"coupled": 1}),
        ("batch_draw_1_ratio83", ds[1], 4, BATCH_OPTS, BATCH_REF),
        ("batch_draw_9_ratio57", ds[9], 4, BATCH_OPTS, BATCH_REF),
        ("drop_256x512", W.rising_drop_256x512(), 2, {"precision": 1}, {}),
        ("drop_256x512_wavefront", W.rising_drop_256x512(), 2,
         {"precision": 1, "wave_cells32": 1}, {}),
        ("drop_256x512_coupled", W.rising_drop_256x512(), 2, {"precision": 1, "coupled": 1},
         {"coupled": 1}),
        ("drop_512_coupled", _drop512(), 1, {"precision": 1, "coupled": 1}, {"coupled": 1}),
    ]


CASES = _cases()


@pytest.mark.parametrize("name,P,steps,gopts,ropts", CASES, ids=[c[0] for c in CASES])
def test_mixed_step_against_the_oracle(qn, name, P, steps, gopts, ropts):
    if name.startswith("batch_draw"):
        ratio = max(P.rho1, P.rho2) / min(P.rho1, P.rho2)
        assert ratio >= 50.0, ratio
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **gopts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **ropts)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    m0 = r.mass()
    for _ in range(steps):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert resg <= P.tol and resr <= P.tol
        assert abs(ng - nr) <= 1, (ng, nr)
    check_mixed(g.get_fields(), r.get_fields())
    mg = g.mass()
    assert abs(mg[0] - m0[0]) <= MIXED_MASS_TOL * m0[0]
    assert abs(mg[1] - m0[1]) <= MIXED_MASS_TOL * m0[1]


def test_fp64_full_size_three_steps_after_five(qn):
    """The benchmark workload past its start: the GPU's state after five FP64
    steps, then three more steps on the GPU and in the oracle from that state:
    equal V-cycle counts and every field within 1e-10."""
    P = W.rising_drop_256x512()
    g = qn.Solver(**P.create_kwargs(), tol=P.tol)
    g.set_fields(P.fields())
    for _ in range(5):
        g.step(P.dt)
    start = g.get_fields()
    r = RefSolver(**P.create_kwargs(), tol=P.tol)
    r.set_fields(start)
    for _ in range(3):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert ng == nr and resg <= P.tol and resr <= P.tol
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        e = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
        assert e <= 1e-10, (k, e)
    mg, mr = g.mass(), r.mass()
    assert abs(mg[0] - mr[0]) <= 1e-13 * mr[0] and abs(mg[1] - mr[1]) <= 1e-13 * mr[1]


def _bench():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "bench.py")
    spec = importlib.util.spec_from_file_location("bench_for_parity", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


# the bench's paths on its workload with the options it times them with
# (bench.PATH_OPTIONS: smoothing counts and predictor), the oracle running the
# same options and smoother
BENCH_PATHS = [
    ("fp64", {}, {}),
    ("mixed", {"precision": 1}, {}),
    ("fp64_coupled", {"coupled": 1}, {"coupled": 1}),
    ("mixed_coupled", {"precision": 1, "coupled": 1}, {"coupled": 1}),
    ("projection_fp64", {"scheme": 1}, {"scheme": 1}),
]


@pytest.mark.parametrize("name,gopts,ropts", BENCH_PATHS, ids=[c[0] for c in BENCH_PATHS])
def test_bench_paths_with_their_options(qn, name, gopts, ropts):
    """Four steps of the 256x512 drop per path (the last two start from the
    predicted iterate): FP64 paths with equal V-cycle counts and every field
    within 1e-10 of the oracle, mixed paths within the mixed bars and one
    V-cycle."""
    nu = _bench().PATH_OPTIONS[name]
    P = W.rising_drop_256x512()
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **gopts, **nu)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **ropts, **nu)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    mixed = gopts.get("precision", 0) == 1
    for _ in range(4):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert resg <= P.tol and resr <= P.tol
        assert (abs(ng - nr) <= 1) if mixed else (ng == nr), (ng, nr)
    fg, fr = g.get_fields(), r.get_fields()
    if mixed:
        check_mixed(fg, fr)
    else:
        for k in fg:
            e = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
            assert e <= 1e-10, (k, e)
