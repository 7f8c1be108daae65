"""ctypes binding of libqnsch_probe.so: the FMA throughput and FP64 issue-cost
probes (csrc/probe.cu).  Measurement tooling, not part of the solver's ABI:
bench.py takes the FP64 peak of its ALU roofline from fma_probe, run in the
same process as the kernels it divides, and profile_kernels prints both."""
from __future__ import annotations

import ctypes
import os

from . import build as _build
from .qnsch import QnschError

_lib = None


def lib():
    """Load (building first if stale) the in-tree libqnsch_probe.so."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.PROBE_LIB) or _build.is_stale():
            _build.build()
        L = ctypes.CDLL(_build.PROBE_LIB)
        i, p = ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        L.qnsch_fma_probe.argtypes = [i, i, i, p]
        L.qnsch_fp64_issue_probe.argtypes = [i, i, i, i, p]
        L.qnsch_stage_probe.argtypes = [i, i, i, i, i, p]
        L.qnsch_rcp_check.argtypes = [i, p, p, p]
        _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        raise QnschError(what, rc)


def fma_probe(fp64=True, blocks_per_sm=8, iters=4096):
    """qnsch_fma_probe: FMA throughput of the current device in TFLOP/s (FP64
    or FP32), the denominator of the FP64 kernels' ALU roofline."""
    t = ctypes.c_double()
    _check(lib().qnsch_fma_probe(int(bool(fp64)), int(blocks_per_sm), int(iters),
                                 ctypes.byref(t)), "qnsch_fma_probe")
    return t.value


def fp64_issue_probe(warps_per_block=4, active_lanes=32, chains=8, iters=1024):
    """qnsch_fp64_issue_probe: SM cycles one warp-wide FP64 FMA holds a
    sub-partition for, with `active_lanes` lanes and `chains` independent
    chains per lane."""
    t = ctypes.c_double()
    _check(lib().qnsch_fp64_issue_probe(int(warps_per_block), int(active_lanes), int(chains),
                                        int(iters), ctypes.byref(t)), "qnsch_fp64_issue_probe")
    return t.value


def stage_probe(mode, threads=128, nb=152, K=0, stages=200):
    """qnsch_stage_probe: microseconds per dependent stage, mode 0 = stages
    separated by an inter-block barrier inside one cooperative launch, mode 1 =
    one launch per stage in a CUDA graph with programmatic dependent launch."""
    t = ctypes.c_double()
    _check(lib().qnsch_stage_probe(int(mode), int(threads), int(nb), int(K), int(stages),
                                   ctypes.byref(t)), "qnsch_stage_probe")
    return t.value


def rcp_check(x):
    """qnsch_rcp_check: (the block solves' FP64 reciprocal of x, IEEE 1/x),
    both computed on the device, for a float64 numpy array x."""
    import numpy as np
    x = np.ascontiguousarray(x, dtype=np.float64)
    yf, yi = np.empty_like(x), np.empty_like(x)
    _check(lib().qnsch_rcp_check(int(x.size), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 yf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 yi.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "qnsch_rcp_check")
    return yf, yi


def fp64_peak_tflops():
    """The best FP64 rate of the throughput probe over 4, 8 and 16 blocks per
    SM (the launch shapes profile_kernels --kernel fmapeak reports)."""
    return max(fma_probe(True, b, 1024) for b in (4, 8, 16))
