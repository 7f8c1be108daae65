"""The fused V-cycle of the small levels as one thread-block cluster (option
fuse_ctas) against the same V-cycle in one thread block, against the per-level
launches, and against the FP64 oracle.

The cluster runs the same device code per cell in the same colour order as the
single block; only which threads take which visits changes (a larger group can
give four-lane teams to larger colours), so FP64 iterates agree to rounding and
full steps match the oracle to 1e-10 with equal V-cycle counts."""
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


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def same_fields(fg, fr, tol, keys=("c", "mu", "p", "u", "v")):
    for k in keys:
        e = relerr(fg[k], fr[k])
        assert e <= tol, (k, e)


def test_cluster_size_option(qn):
    """fuse_ctas takes a power of two from 1 to 16; the handle keeps the
    largest size not above it that the device launches (at least 8, the
    portable cluster size, on this GPU); other values are refused and leave
    the option unchanged."""
    P = W.small_case(32, 32, True)
    g = qn.Solver(**P.create_kwargs())
    assert g.get_option("fuse_ctas") == 1
    for bad in (0, 3, 6, 17, 32, -1, 2.5):
        with pytest.raises(qn.QnschError):
            g.set_option("fuse_ctas", bad)
        assert g.get_option("fuse_ctas") == 1
    for want in (2, 4, 8, 16):
        g.set_option("fuse_ctas", want)
        got = g.get_option("fuse_ctas")
        assert got <= want and int(got) & (int(got) - 1) == 0
        assert got >= min(want, 8)


@pytest.mark.parametrize("precision,px,coupled",
                         [(0, False, 0), (0, True, 0), (1, False, 0), (1, True, 0),
                          (0, False, 1), (1, False, 1)])
def test_cluster_vcycle_matches_block_and_per_level_launches(qn, precision, px, coupled):
    """Two V-cycles with every level fused, in one block and in clusters of
    2, 4, 8 and 16 blocks, and with no level fused: the iterates agree to
    rounding (FP64), or to the FP32 error cycle's rounding (mixed)."""
    P = W.small_case(64, 96, px)
    f = P.fields()
    out = {}
    for fuse, ctas in ((0, 1), (10 ** 6, 1), (10 ** 6, 2), (10 ** 6, 4), (10 ** 6, 8),
                       (10 ** 6, 16)):
        g = qn.Solver(**P.create_kwargs(), precision=precision, coupled=coupled,
                      fuse_cells=fuse, fuse_cells32=fuse, fuse_ctas=ctas)
        g.set_fields(f)
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out[(fuse, ctas)] = g.get_iterate()
    tol = 1e-12 if precision == 0 else 1e-5
    ref = out[(10 ** 6, 1)]
    for key, it in out.items():
        same_fields(it, ref, tol)


def test_cluster_projection_vcycle_matches_block(qn):
    """The projection method's fused smoother (CH, four-velocity blocks,
    pressure Gauss-Seidel) in a 16-block cluster equals the single block."""
    P = W.small_case(64, 64, False)
    f = P.fields()
    out = []
    for ctas in (1, 16):
        g = qn.Solver(**P.create_kwargs(), scheme=1, fuse_cells=10 ** 6, fuse_ctas=ctas)
        g.set_fields(f)
        g.begin_step(P.dt)
        for _ in range(2):
            g.vcycle()
        out.append(g.get_iterate())
    same_fields(out[1], out[0], 1e-12)


@pytest.mark.parametrize("m1,m2,px,opts", [
    (64, 128, False, {}),
    (96, 64, True, {}),
    (64, 128, False, {"coupled": 1}),
    (64, 64, False, {"scheme": 1}),
])
def test_cluster_steps_match_oracle(qn, m1, m2, px, opts):
    """Three FP64 steps with the levels up to 2048 cells fused in a 16-block
    cluster: equal V-cycle counts and every field within 1e-10 of the oracle."""
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs(), tol=1e-10, fuse_cells=2048, fuse_ctas=16, **opts)
    r = RefSolver(**P.create_kwargs(), tol=1e-10, **opts)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    for _ in range(3):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert ng == nr and resg <= 1e-10 and resr <= 1e-10, (ng, nr)
    same_fields(g.get_fields(), r.get_fields(), 1e-10)


def test_cluster_mixed_steps_meet_mixed_bars(qn):
    """Mixed precision with the FP32 levels up to 8192 cells fused in a
    16-block cluster: the FP64 tolerance is met and the fields stay within the
    mixed-precision bars of the oracle."""
    P = W.small_case(128, 128, True)
    g = qn.Solver(**P.create_kwargs(), tol=1e-9, precision=1, fuse_cells32=8192, fuse_ctas=16)
    r = RefSolver(**P.create_kwargs(), tol=1e-9)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    for _ in range(2):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert resg <= 1e-9 and abs(ng - nr) <= 1, (ng, nr)
    check_mixed(g.get_fields(), r.get_fields())


def test_cluster_rising_drop_full_size(qn):
    """The 256x512 drop with the levels up to 32x64 fused in a 16-block
    cluster and the headline's smoothing counts and predictor: four steps with
    the oracle's V-cycle counts and every field within 1e-10."""
    P = W.rising_drop_256x512()
    nu = {"nu1": 1, "nu2": 1, "nu1_fine": 2, "nu2_fine": 3, "predictor": 2}
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, fuse_cells=2048, fuse_ctas=16, **nu)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **nu)
    f = P.fields()
    g.set_fields(f)
    r.set_fields(f)
    for _ in range(4):
        ng, resg = g.step(P.dt)
        nr, resr = r.step(P.dt)
        assert ng == nr and resg <= P.tol, (ng, nr)
    same_fields(g.get_fields(), r.get_fields(), 1e-10)
