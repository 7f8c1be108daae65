"""The FMA probes behind the FP64 cost model (libqnsch_probe.so, measurement
tooling beside the solver library): the throughput probe (the FP64
kernels' ALU-roofline peak) runs and its rates are of the right order (FP32
far above FP64 on a part whose FP64 rate is a small fraction of its FP32
rate); the issue-cost probe gives a positive, finite cycle count per warp FMA
that does not fall when lanes go idle (the pipe's cost is per warp
instruction, not per active lane)."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rates():
    from paper_1703_06606_gb300 import probe
    f64 = probe.fma_probe(True, 4, 256)
    f32 = probe.fma_probe(False, 4, 256)
    assert 0.05 < f64 < 100.0, f64
    assert f32 > 5.0 * f64, (f32, f64)


def test_fp64_issue_probe_cost_is_per_warp_instruction():
    from paper_1703_06606_gb300 import probe
    full = probe.fp64_issue_probe(4, 32, 8, 64)
    one = probe.fp64_issue_probe(4, 1, 8, 64)
    assert math.isfinite(full) and 1.0 < full < 1000.0, full
    # a per-active-lane cost would make `one` about full / 32
    assert one > 0.25 * full, (one, full)


def test_stage_probe_both_forms_run():
    """The stage probe's two forms (inter-block barrier in one cooperative
    launch; one graph-captured launch per stage) both finish, with positive,
    finite costs per stage that grow with the FP64 chain each stage runs."""
    from paper_1703_06606_gb300 import probe
    for mode in (0, 1):
        empty = probe.stage_probe(mode, 128, 8, 0, 50)
        chain = probe.stage_probe(mode, 128, 8, 64, 50)
        assert math.isfinite(empty) and 0.0 < empty < 100.0, (mode, empty)
        assert chain > empty, (mode, chain, empty)


def test_block_solve_reciprocal_is_within_two_ulp_of_ieee_division():
    """The FP64 reciprocal of the local block solves (Newton-Raphson from the
    hardware's approximate reciprocal) against IEEE 1/x on the device, over
    magnitudes from 1e-200 to 1e200 of both signs: at most 2 units in the last
    place apart, and exact on powers of two."""
    import numpy as np
    from paper_1703_06606_gb300 import probe
    rng = np.random.default_rng(1703066)
    x = np.exp(rng.uniform(np.log(1e-200), np.log(1e200), 200000))
    x *= np.where(rng.random(x.size) < 0.5, -1.0, 1.0)
    x = np.concatenate([x, 2.0 ** np.arange(-60, 61), [1.0, 3.0, 7.0, 0.1]])
    yf, yi = probe.rcp_check(x)
    ulp = np.abs(yf - yi) / np.spacing(np.abs(yi))
    assert np.all(np.isfinite(yf)) and ulp.max() <= 2.0, ulp.max()
    p2 = 2.0 ** np.arange(-60, 61)
    yf2, _ = probe.rcp_check(p2)
    assert np.array_equal(yf2, 1.0 / p2)
