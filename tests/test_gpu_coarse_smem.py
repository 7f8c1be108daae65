"""The fused coarse V-cycle of the FP64 levels on a shared-memory copy of its
levels (option coarse_smem, on by default): the same device code on the same
values as the launch that reads global memory, so V-cycles give bitwise the
same fields; against the FP64 oracle the V-cycles and full droplet steps keep
their 1e-10 bar and equal V-cycle counts; a fused group whose copy does not
fit falls back to global memory."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("m1,m2,px,coupled", [(64, 96, False, 0), (64, 64, True, 0),
                                              (48, 80, False, 1), (40, 40, True, 0)])
def test_shared_copy_matches_global_bitwise(qn, m1, m2, px, coupled):
    P = W.small_case(m1, m2, px)
    a = qn.Solver(**P.create_kwargs(), coarse_smem=1, coupled=coupled)
    b = qn.Solver(**P.create_kwargs(), coarse_smem=0, coupled=coupled)
    for s in (a, b):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        na, nb = a.vcycle(), b.vcycle()
        assert np.array_equal(na, nb)
    assert a.get_option("coarse_smem_used") == 1
    assert b.get_option("coarse_smem_used") == 0
    fa, fb = a.get_iterate(), b.get_iterate()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


@pytest.mark.parametrize("m1,m2,px", [(32, 48, False), (64, 96, True)])
def test_shared_copy_vcycle_parity(qn, m1, m2, px):
    P = W.small_case(m1, m2, px)
    g = qn.Solver(**P.create_kwargs(), coarse_smem=1)
    r = RefSolver(**P.create_kwargs())
    for s in (g, r):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
    for _ in range(3):
        g.vcycle()
        r.vcycle()
        assert g.get_option("coarse_smem_used") == 1
        fg, fr = g.get_iterate(), r.get_iterate()
        for k in fg:
            assert relerr(fg[k], fr[k]) <= 1e-10, k


def test_shared_copy_full_steps_rising_drop(qn):
    """Three steps of the 256x512 droplet with the headline's options: the
    fused 8x16, 4x8 and 2x4 levels run from shared memory; equal V-cycle
    counts and fields within 1e-10 of the oracle."""
    P = W.rising_drop_256x512()
    opts = dict(nu1=1, nu2=1, nu1_fine=2, nu2_fine=3, predictor=2)
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, coarse_smem=1, **opts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **opts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    for _ in range(3):
        ng, _ = g.step(P.dt)
        nr, _ = r.step(P.dt)
        assert ng == nr
        assert g.get_option("coarse_smem_used") == 1
    fg, fr = g.get_fields(), r.get_fields()
    for k in fg:
        assert relerr(fg[k], fr[k]) <= 1e-10, k


def test_group_too_wide_for_the_copy_falls_back(qn):
    """fuse_cells = 512 puts the 16x32 level of the droplet into the fused
    group; its rows (35 padded cells) are wider than the copy's 32-column
    rows, so the launch reads global memory and the results are unchanged."""
    P = W.rising_drop_256x512()
    a = qn.Solver(**P.create_kwargs(), fuse_cells=512, coarse_smem=1)
    b = qn.Solver(**P.create_kwargs(), fuse_cells=512, coarse_smem=0)
    for s in (a, b):
        s.set_fields(P.fields())
        s.begin_step(P.dt)
        s.vcycle()
    assert a.get_option("coarse_smem_used") == 0
    fa, fb = a.get_iterate(), b.get_iterate()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
