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
