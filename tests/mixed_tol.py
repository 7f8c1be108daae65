"""The mixed-precision parity bar: per field, the largest relative max-norm
difference between a mixed-precision GPU step (FP32 FAS cycles on the error
equation under the FP64 defect correction) and the FP64 oracle's step from the
same state, both converged to the same FP64 residual tolerance.

The bar is about ten times the largest difference measured on a GB300 over
the parity cases of tests/test_gpu_mixed_parity.py (small wall-bounded and
periodic cases, both smoothers, the 64^2 and 128^2 batch draws at density
ratios 83 and 57 with the batch's launch options, the 256x512 rising drop and a
512^2 drop with the coupled block): c 3.4e-16, mu 5.6e-13, p 3.1e-13,
u 1.41e-12, v 1.37e-12.  The FP64 defect correction decides the answer; the
FP32 cycle only has to reduce the error, so these differences are the FP64
discretisation's sensitivity at the stopping tolerance, not FP32 rounding.
Mass (sum rho, sum rho c) drifts by at most 3.0e-13 relative per step."""

MIXED_TOL = {"c": 5e-15, "mu": 6e-12, "p": 3e-12, "u": 1.5e-11, "v": 1.5e-11}
MIXED_MASS_TOL = 3e-12


def check_mixed(fg, fr):
    """Assert every field of fg within its bar of fr; returns the errors."""
    import numpy as np
    errs = {}
    for k, tol in MIXED_TOL.items():
        e = float(np.max(np.abs(fg[k] - fr[k])) / max(np.max(np.abs(fr[k])), 1e-300))
        errs[k] = e
        assert e <= tol, (k, e, tol)
    return errs
