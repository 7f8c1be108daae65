"""Run single kernels of libqnsch.so on a chosen grid, for profilers (ncu).

    python -m paper_1703_06606_gb300.profile_kernels --kernel vanka --m1 1024 --m2 1024 --reps 3
    python -m paper_1703_06606_gb300.profile_kernels --workload rt --kernel step --precision 1
    python -m paper_1703_06606_gb300.profile_kernels --workload rt --kernel step --precision 1 \
        --option skew_cells32=1048576 --option skew_rows=64
    python -m paper_1703_06606_gb300.profile_kernels --kernel fmapeak
    python -m paper_1703_06606_gb300.profile_kernels --kernel fp64issue
    python -m paper_1703_06606_gb300.profile_kernels --kernel stage

Sets up the drop workload at the given size (default 1024 x 1024), or the
Rayleigh-Taylor workload at its full 1024 x 4096 size, freezes a time step
and issues `reps` launches of one finest-level kernel (vanka: colour 0 of the
Vanka smoother; ch: colour 0 of the CH smoother; residual: the residual and
its norms; step: whole time steps, in the FP64 (--precision 0) or mixed
(--precision 1) path, with the paper's smoother or the coupled block
(--coupled 1), or the projection method (--scheme 1)).  fmapeak times the
FMA throughput probe of libqnsch_probe.so (qnsch_fma_probe) in FP64 and FP32 over a few
launch shapes and prints the rates; the best FP64 rate is the peak of the
FP64 kernels' ALU roofline.  fp64issue runs qnsch_fp64_issue_probe over active
lanes, independent chains and warps per block and prints the SM cycles one
warp-wide FP64 FMA holds a sub-partition for.  stage runs qnsch_stage_probe
and prints the cost of one dependent stage when stages are separated by an
inter-block barrier inside one cooperative launch and when each stage is its
own graph-captured launch with programmatic dependent launch, over the blocks
that take part and the FP64 chain each stage runs.
"""
from __future__ import annotations

import argparse

from . import probe, qnsch, workloads


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", default="vanka", choices=["vanka", "ch", "residual", "step", "fmapeak",
                                                              "fp64issue", "stage"])
    ap.add_argument("--workload", default="drop", choices=["drop", "rt"])
    ap.add_argument("--m1", type=int, default=1024)
    ap.add_argument("--m2", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--coupled", type=int, default=0, choices=[0, 1])
    ap.add_argument("--scheme", type=int, default=0, choices=[0, 1])
    ap.add_argument("--option", action="append", default=[], metavar="KEY=VALUE",
                    help="a solver option for the step (repeatable), e.g. skew_cells32=1048576")
    a = ap.parse_args()
    if a.kernel == "fmapeak":
        for fp64 in (True, False):
            rates = {b: probe.fma_probe(fp64, b, 1024) for b in (4, 8, 16)}
            for b, r in rates.items():
                print("%s blocks/SM %2d: %.4f TFLOP/s" % ("FP64" if fp64 else "FP32", b, r))
            print("%s best: %.4f TFLOP/s" % ("FP64" if fp64 else "FP32", max(rates.values())))
        return
    if a.kernel == "fp64issue":
        print("warps/block  active lanes  chains  cycles per warp FMA")
        for warps in (1, 2, 3, 4, 8, 16):
            for active in (1, 32):
                for chains in (1, 8):
                    c = probe.fp64_issue_probe(warps, active, chains, 1024)
                    print("%11d  %12d  %6d  %.1f" % (warps, active, chains, c))
        return
    if a.kernel == "stage":
        print("threads  blocks  FP64 chain  us/stage barrier  us/stage graph launches")
        for threads in (128, 256):
            for K in (0, 64):
                for nb in (152, 64, 16, 4, 1):
                    b = probe.stage_probe(0, threads, nb, K, 200)
                    g = probe.stage_probe(1, threads, nb, K, 200)
                    print("%7d  %6d  %10d  %16.3f  %23.3f" % (threads, nb, K, b, g))
        return
    if a.workload == "rt":
        P = workloads.rayleigh_taylor_1024x4096()
    else:
        P = workloads.rising_drop_256x512()
        P.m1, P.m2, P.Lx = a.m1, a.m2, 1.0
        P.init_args = dict(x0=0.5, y0=0.25 * a.m2 / a.m1, R=0.2)
    opts = {}
    for kv in a.option:
        k, v = kv.split("=", 1)
        opts[k] = float(v)
    s = qnsch.Solver(**P.create_kwargs(), tol=P.tol, precision=a.precision, coupled=a.coupled,
                     scheme=a.scheme, **opts)
    s.set_fields(P.fields())
    if a.kernel == "step":
        for _ in range(a.reps):
            print(s.step(P.dt))
        return
    s.begin_step(P.dt)
    for _ in range(a.reps):
        if a.kernel == "vanka":
            s.smooth_vanka(0)
        elif a.kernel == "ch":
            s.smooth_ch(0)
        else:
            s.residual()
    print("done", a)


if __name__ == "__main__":
    main()
