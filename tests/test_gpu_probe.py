"""The FMA throughput probe that gives the FP64 kernels' ALU-roofline peak:
it runs, and its rates are of the right order (FP32 far above FP64 on a part
whose FP64 rate is a small fraction of its FP32 rate)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_probe_rates():
    from paper_1703_06606_gb300 import qnsch
    f64 = qnsch.fma_probe(True, 4, 256)
    f32 = qnsch.fma_probe(False, 4, 256)
    assert 0.05 < f64 < 100.0, f64
    assert f32 > 5.0 * f64, (f32, f64)
