"""qnsch_mass_noalloc: the mass reduction for callers that must not allocate.

Code that runs inside an allocator or memory-pool callback, under a
device-memory budget that another framework has reserved in full, or in a loop
that must not synchronise the device cannot call cudaMalloc when it needs a
result.  qnsch_mass_noalloc serves them: it reads the caller's array,
writes the caller's output and keeps its scratch in a fixed device array of the
library.  This test checks it, through the C ABI, against the handle-based
qnsch_mass on the same fields, on two consecutive calls (the second call must
not depend on what the first left in the shared scratch).

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes when run alone.
"""
import numpy as np
import pytest

from paper_1703_06606_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1703_06606_gb300 import qnsch
    return torch, qnsch


def test_noalloc_mass_matches_handle_mass_on_two_calls(env):
    torch, qnsch = env
    cases = [(W.small_case(64, 48, False, rho_ratio=10.0), 11),
             (W.rising_drop_256x512(), 12)]
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for P, seed in cases:
        f = W.random_state(P.m1, P.m2, P.periodic_x, seed=seed)
        g = qnsch.Solver(**P.create_kwargs())
        g.set_fields(f)
        want = np.array(g.mass())
        c = torch.tensor(f["c"], dtype=torch.float64, device="cuda")
        for _ in range(2):
            out.fill_(float("nan"))
            qnsch.mass_noalloc(c, P.h, P.rho1, P.rho2, out, stream=stream)
            stream.synchronize()
            got = out.cpu().numpy()
            assert np.allclose(got, want, rtol=1e-12, atol=0), (got, want)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, qnsch = env
    c = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    lib = qnsch.lib()
    # 4096 x 4096 cells exceed QNSCH_NOALLOC_MAX_CELLS: rejected before any launch
    rc = lib.qnsch_mass_noalloc(c.data_ptr(), 4096, 4096, 1.0, 1.0, 2.0, out.data_ptr(), None)
    assert rc == -1
