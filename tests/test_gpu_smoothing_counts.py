"""The finest level's own smoothing counts (nu1_fine, nu2_fine) on the GPU
against the oracle with the same options: equal V-cycle counts and every field
within 1e-10 (FP64), within the mixed bars (mixed precision), for the paper's
smoother, the coupled block and the projection method.  A finest level with
counts of its own is kept out of the single-block coarse V-cycle, so grids
whose finest level would be fused (16 x 16 with the fused threshold above it)
follow the oracle too."""
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


def _counts(fine, coarse):
    return {"nu1": coarse[0], "nu2": coarse[1], "nu1_fine": fine[0], "nu2_fine": fine[1]}


CASES = [
    ("walls_fp64", W.small_case(32, 48, False), _counts((2, 3), (1, 1)), {}, {}),
    ("periodic_fp64", W.small_case(32, 32, True), _counts((3, 2), (1, 1)), {}, {}),
    ("coupled_fp64", W.small_case(32, 48, False), _counts((1, 3), (1, 1)), {"coupled": 1},
     {"coupled": 1}),
    ("projection_fp64", W.small_case(32, 64, False), _counts((2, 2), (1, 1)), {"scheme": 1},
     {"scheme": 1}),
    ("fused_finest_fp64", W.small_case(16, 16, False), _counts((3, 2), (1, 1)),
     {"fuse_cells": 4096}, {}),
    ("mixed", W.small_case(64, 48, False, rho_ratio=10.0), _counts((2, 3), (1, 1)),
     {"precision": 1}, {}),
    ("fused_finest_mixed", W.small_case(16, 16, True), _counts((2, 3), (1, 1)),
     {"precision": 1, "fuse_cells32": 4096}, {}),
]


@pytest.mark.parametrize("name,P,counts,gopts,ropts", CASES, ids=[c[0] for c in CASES])
def test_fine_counts_match_the_oracle(qn, name, P, counts, gopts, ropts):
    g = qn.Solver(**P.create_kwargs(), tol=P.tol, **counts, **gopts)
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **counts, **ropts)
    g.set_fields(P.fields())
    r.set_fields(P.fields())
    mixed = gopts.get("precision", 0) == 1
    for _ in range(3):
        ng, rg = g.step(P.dt)
        nr, rr = r.step(P.dt)
        assert rg <= P.tol and rr <= P.tol
        assert (abs(ng - nr) <= 1) if mixed else (ng == nr), (ng, nr)
    fg, fr = g.get_fields(), r.get_fields()
    if mixed:
        check_mixed(fg, fr)
    else:
        for k in fg:
            e = np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300)
            assert e <= 1e-10, (k, e)
