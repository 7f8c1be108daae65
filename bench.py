"""Benchmark: cell-updates per second of the implicit primitive q-NSCH time step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One "step" is one implicit time step of the primitive method (Sec. 6.1 of
arXiv:1703.06606): freeze the level-n data on every multigrid level, run FAS
V-cycles (Sec. 7.1) until the largest scaled residual norm is <= 1e-9, commit.
Workload: the rising droplet, 256 x 512 cells on [0,1] x [0,2], walls all round,
drop radius 0.25 at (0.5, 0.5), rho and viscosity ratio 10 (light drop),
Re = 35, We = 10, Fr = 1, Cn = 0.01, dt = 2e-4, FP64 (synthetic initial state,
no dataset).  value = cells x K / (device time of the K timed steps), inputs
resident in HBM; L2 is flushed (256 MiB write) between timed steps.

With N > 1 (torchrun) each rank runs an independent replica of the workload on
its own GPU (a single instance does not shard); value sums the cells of all
ranks over the slowest rank's time.

--impl reference times the FP64 CPU oracle (serial C, host cores) on the same
workload and prints the same JSON line with "impl": "reference".

cpu_baseline is the serial oracle on a few steps of the workload;
cpu_baseline.all_cores runs one independent oracle replica per host core
(spawned processes, started together) for the whole-job CPU throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1703_06606_gb300 import replicas, workloads  # noqa: E402

METRIC = ("cell-updates/s per time step at residual 1e-9 (FP64 plain vs batched mixed) "
          "+ p99 latency")
UNIT = "cell-updates/s"


def field_bytes(P):
    m1, m2 = P.m1, P.m2
    return 8 * (3 * m1 * m2 + (m1 + 1) * m2 + m1 * (m2 + 1))


# Solver options per path: the smoothing steps before (nu1) and after (nu2)
# the coarse-grid correction, and the predicted initial iterate (predictor).
# The paper leaves both open.  The library's and the oracle's defaults are the
# reading: nu1 = nu2 = 2, and each step starts from x^n.  The bench runs each
# path with the options measured fastest on a GB300 at its own protocol (ms per
# step over 20 steps after 5 warm-up, the 256x512 drop unless named;
# nu_coarse 4 throughout):
#   FP64, the paper's smoother: (3, 2) with the quadratic predictor 20.4,
#     against (3, 2) 28.7 and (2, 2) 31.3 without a predictor, (3, 2) with
#     the linear one 23.9, (2, 2) with the quadratic one 20.6
#   mixed, the paper's smoother: (3, 2) quadratic 8.7, against (3, 1) 12.4
#     and (2, 2) 13.4 without, (3, 1) quadratic 9.1
#   FP64 coupled: (1, 2) quadratic 15.5, against (1, 2) 19.1 and (2, 2) 24.1
#     without
#   mixed coupled: (1, 2) quadratic 5.7, against (1, 2) 6.9 and (2, 2) 8.2
#     without
#   projection, FP64: (1, 2) quadratic 18.8, against (1, 2) 19.8 and (2, 2)
#     22.3 without
#   capillary wave 64^2, FP64: (3, 2) quadratic 3.0, against (3, 2) 5.7 and
#     (2, 2) 6.4 without
#   Rayleigh-Taylor 1024x4096, mixed (5 steps after 5 warm-up): (1, 2)
#     quadratic 19.7, against (1, 2) 49.3 without; its first steps move fast
#     (the interface relaxes), and there extrapolation costs cycles, so the
#     workload is timed after 5 warm-up steps
# and then, with the quadratic predictor, counts of the finest level's own
# (nu1_fine, nu2_fine) over one step each below it (nu1 = nu2 = 1):
#   FP64, the paper's smoother: finest (2, 3) 14.7 (7.4 V-cycles), (3, 2)
#     15.2, (2, 4) 15.1, (3, 3) 15.4, against (3, 2) on every level 20.5;
#     below (2, 2) 18.6 and (2, 1) 16.7 with the finest at (3, 2)
#   mixed, the paper's smoother: finest (2, 3) 6.3, (3, 2) 6.5, against
#     (3, 2) on every level 8.8
#   capillary wave: finest (3, 2) 2.6 against 3.7 on every level
#   coupled and projection paths, RT: no gain (already (1, 2) everywhere)
# Every step still stops at the same FP64 residual tolerance.  The oracle legs
# (cpu_baseline, --impl reference) run the headline's options, and the
# cpu_baseline starts from the GPU's state and history, so that both time the
# same V-cycles.  The stress cases and the Sec. 9 table keep the defaults.
PATH_OPTIONS = {
    "fp64": {"nu1": 1, "nu2": 1, "nu1_fine": 2, "nu2_fine": 3, "predictor": 2},
    "mixed": {"nu1": 1, "nu2": 1, "nu1_fine": 2, "nu2_fine": 3, "predictor": 2},
    "fp64_coupled": {"nu1": 1, "nu2": 2, "predictor": 2},
    "mixed_coupled": {"nu1": 1, "nu2": 2, "predictor": 2},
    "projection_fp64": {"nu1": 1, "nu2": 2, "predictor": 2},
    "fp64_device_loop": {"nu1": 1, "nu2": 1, "nu1_fine": 2, "nu2_fine": 3, "predictor": 2},
    "capillary_wave_64x64": {"nu1": 1, "nu2": 1, "nu1_fine": 3, "nu2_fine": 2, "predictor": 2},
    "rayleigh_taylor_1024x4096": {"nu1": 1, "nu2": 2, "predictor": 2},
}


def config_of(P, levels, precision="fp64", opts=None):
    opts = opts or PATH_OPTIONS["fp64"]
    return {"workload": P.name, "grid": "%dx%d" % (P.m1, P.m2), "levels": levels,
            "dt": P.dt, "tol": P.tol, "precision": precision,
            "smoother": "CH 2x2 red-black + Vanka 5x5 (5 colours)",
            "smoothing_steps": {"finest": [opts.get("nu1_fine", opts["nu1"]),
                                           opts.get("nu2_fine", opts["nu2"])],
                                "below": [opts["nu1"], opts["nu2"]], "coarsest": 4},
            "predictor": "quadratic extrapolation in time of the initial iterate"
                         if opts.get("predictor") == 2 else opts.get("predictor", 0),
            "l2": "flushed between timed steps (256 MiB write)",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, interval_ms=50):
        # 50 ms: the headline's timed region lasts about 0.3 s, so a 200 ms
        # interval left one sample in it
        self.index = index
        self.interval_ms = int(interval_ms)
        self.proc = None
        self.lines = []
        self.first = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", str(self.interval_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def ready(self, timeout_s=10.0):
        """Wait for the sampler's first line (its start-up queries the driver,
        which should not fall inside the timed region); samples from here on
        are the ones summarised."""
        t0 = time.perf_counter()
        while self.proc and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)
        self.first = len(self.lines)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[self.first:] or self.lines[-1:]
        for ln in lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def paper_table2():
    """The paper's Table 2 (Sec. 9), CPU seconds per step of the primitive and
    the projection method by m, as printed (tests/golden/paper_tables_sec9.txt)."""
    prim, proj = {}, {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests", "golden",
                        "paper_tables_sec9.txt")
    with open(path) as f:
        for ln in f:
            w = ln.split()
            if w and w[0] == "table2":
                prim[int(w[1])], proj[int(w[1])] = float(w[2]), float(w[3])
    return prim, proj


# ---------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def host_cpu():
    """The host the CPU baselines ran on: architecture, CPU model (lscpu, else
    /proc/cpuinfo) and logical cores."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        model = next((ln.split(":", 1)[1].strip() for ln in out.splitlines()
                      if ln.lower().startswith("model name")), None)
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                model = next((ln.split(":", 1)[1].strip() for ln in f
                              if ln.lower().startswith("model name")), None)
        except OSError:
            pass
    return {"arch": platform.machine(), "model": model, "nproc": os.cpu_count(),
            "usable": usable_cores(cap=1 << 20)}


def oracle_rate(P, steps, budget_s, fields=None, options=None, history=()):
    """Time the FP64 oracle (serial, as it stands) on the workload: up to `steps`
    implicit steps from `fields` (default: the initial state), stopping once
    `budget_s` is spent; options: the oracle's options (smoothing counts,
    predictor); history: the earlier states the predictor extrapolates from,
    (fields, dt) pairs, the most recent first."""
    from oracle.ref import RefSolver
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **(options or {}))
    r.set_fields(P.fields() if fields is None else fields)
    for k, (hf, hdt) in enumerate(history):
        r.set_history(k, hf, hdt)
    times, cycles = [], []
    t_all = time.perf_counter()
    for _ in range(steps):
        t0 = time.perf_counter()
        n, _ = r.step(P.dt)
        times.append(time.perf_counter() - t0)
        cycles.append(n)
        if time.perf_counter() - t_all > budget_s:
            break
    return times, cycles


def _oracle_replica(workload, steps, barrier, out, options=None):
    """One host core's share of the all-cores oracle baseline: an independent
    oracle instance of `workload` steps `steps` times from its initial state,
    starting together with the other replicas; puts (seconds, V-cycles), or
    None if the start barrier breaks."""
    from oracle.ref import RefSolver
    P = getattr(workloads, workload)()
    r = RefSolver(**P.create_kwargs(), tol=P.tol, **(options or {}))
    r.set_fields(P.fields())
    try:
        barrier.wait(timeout=120)
    except Exception:
        out.put(None)
        return
    cycles = []
    t0 = time.perf_counter()
    for _ in range(steps):
        cycles.append(r.step(P.dt)[0])
    out.put((time.perf_counter() - t0, cycles))


def usable_cores(cap=64):
    """Cores this process may run on (its CPU affinity, which a container's
    cpuset limits), else the machine's count; at most `cap`."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    return max(1, min(n, cap))


def oracle_all_cores(workload="rising_drop_256x512", steps=1, procs=None, timeout=300.0,
                     options=None):
    """Throughput of the FP64 oracle, as it stands, on every host core: one
    independent replica of the workload per core (spawned processes, so no
    CUDA state is inherited), started together; whole-job cell-updates/s =
    replicas x cells x steps / the slowest replica's seconds.  None if a
    replica fails or the run exceeds `timeout`."""
    import multiprocessing as mp
    from oracle.ref import lib as oracle_lib
    oracle_lib()  # compiled once here, before the replicas load it
    n = procs or usable_cores()
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(n), ctx.Queue()
    ps = [ctx.Process(target=_oracle_replica, args=(workload, steps, barrier, out, options),
                      daemon=True)
          for _ in range(n)]
    for p in ps:
        p.start()
    deadline = time.time() + timeout
    res = []
    try:
        for _ in range(n):
            res.append(out.get(timeout=max(1.0, deadline - time.time())))
    except Exception:
        res.append(None)
    for p in ps:
        p.join(timeout=5)
        if p.is_alive():
            p.kill()
    if len(res) != n or any(r is None for r in res):
        return None
    P = getattr(workloads, workload)()
    slowest = max(t for t, _ in res)
    return {"value": n * P.cells * steps / slowest, "unit": UNIT, "cores": n,
            "kind": "oracle replicas",
            "sample": "%d independent serial FP64 oracle instances of %s, one per host core, "
                      "%d step(s) each from the initial state, started together; slowest "
                      "replica %.1f s (V-cycles %s)"
                      % (n, P.name, steps, slowest, "/".join(str(c[0]) for _, c in res[:4]) +
                         ("/..." if n > 4 else ""))}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1703_06606_gb300 import probe, qnsch

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        import torch.distributed as dist
        import datetime
        dist.init_process_group("nccl", device_id=dev,
                                timeout=datetime.timedelta(seconds=replicas.PG_TIMEOUT_S))
    if rank == 0:
        qnsch.lib()  # build once
    if world > 1:
        dist.barrier()
    qnsch.lib()

    P = workloads.rising_drop_256x512()
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    s = qnsch.Solver(**P.create_kwargs(), tol=P.tol, stream=stream, **PATH_OPTIONS["fp64"])
    levels = s.levels
    f0 = P.fields()
    dev_fields = {k: torch.tensor(v, device=dev, dtype=torch.float64) for k, v in f0.items()}
    s.set_fields_device(dev_fields)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        s.step(P.dt)
    torch.cuda.synchronize()
    # the committed state the timed steps start from and the earlier states the
    # predictor extrapolates from (the CPU baseline starts the oracle from
    # them, so both time the same steps)
    start_fields = s.get_fields()
    start_hist = [s.history(k) for k in range(int(s.get_option("history")))]

    # ---- timed region: K steps, device time per step (CUDA events on our
    # stream); each step is one graph whose outer-cycle loop runs on the device
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    cyc = []
    l0 = qnsch.kernel_launches()
    failed = None
    with ClockSampler(local_rank) as clk:
        clk.ready()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        try:
            for k in range(args.steps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                n, res = s.step(P.dt)
                evs[k][1].record(stream)
                cyc.append(n)
        except qnsch.QnschError as e:
            failed = e
        torch.cuda.synchronize()
    if failed is not None:
        print("bench: a timed step failed: %s" % failed, file=sys.stderr, flush=True)
        replicas.slowest(0.0, dev, ok=False)  # every rank stops here
    launches = qnsch.kernel_launches() - l0
    device_loop = s.get_option("device_loop")
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_s = replicas.slowest(sum(step_ms) / 1e3, dev)
    if world > 1:
        dist.barrier()

    # ---- kernel timing by kind on the same workload, right after the timed
    # region: CUDA events around every launch of each kind inside the replayed
    # cycle graphs (the same kernels and launch shapes as the timed steps)
    kinds = prof_kinds(s, P, stream, flush, nsteps=max(2, min(args.steps, 5)))
    fp64_peak = probe.fp64_peak_tflops()

    # ---- the same workload in the other solver variants: mixed precision (FP32
    # FAS cycles on the error equation under FP64 defect correction) and the
    # coupled 7x7 smoother
    variants = {}
    if not args.no_variants:
        for name, prec, coup, sch, extra in (
                ("mixed", 1, 0, 0, {}), ("fp64_coupled", 0, 1, 0, {}),
                ("mixed_coupled", 1, 1, 0, {}), ("projection_fp64", 0, 0, 1, {}),
                ("fp64_device_loop", 0, 0, 0, {"device_loop": 1})):
            extra = dict(extra, **PATH_OPTIONS[name])
            sv = qnsch.Solver(**P.create_kwargs(), tol=P.tol, stream=stream, precision=prec,
                              coupled=coup, scheme=sch, **extra)
            sv.set_fields_device(dev_fields)
            for _ in range(args.warmup):
                sv.step(P.dt)
            vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            vcyc = []
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))
                vev[k][0].record(stream)
                n, res = sv.step(P.dt)
                vev[k][1].record(stream)
                vcyc.append(n)
            torch.cuda.synchronize()
            vms = [a.elapsed_time(b) for a, b in vev]
            vtot = replicas.slowest(sum(vms) / 1e3, dev)
            variants[name] = {
                "value": world * P.cells * args.steps / vtot, "unit": UNIT,
                "ms_per_step": float(np.mean(vms)),
                "latency_ms": {"p50": float(np.percentile(vms, 50)),
                               "p99": float(np.percentile(vms, 99))},
                "vcycles_per_step": float(np.mean(vcyc)), "tol": P.tol,
                "precision": ("FP32 FAS cycles on the error equation; FP64 residual, defect "
                              "correction, gauge, mass, energy") if prec else "FP64",
                "options": extra,
                "smoother": "coupled 7x7 block, 5 colours" if coup else
                            ("projection method (Sec. 6.2): CH 2x2 red-black, intermediate-"
                             "velocity Vanka 4x4 (5 colours), pressure Gauss-Seidel red-black"
                             if sch else "CH 2x2 red-black + Vanka 5x5 (5 colours)")}
            sv.close()

    # ---- high-ratio stress cases: capillary wave at density ratio 1:1000 (256^2)
    # and the droplet with the paper's own parameters (256x512, periodic x),
    # FP64 with the paper's smoother and mixed precision with the coupled block
    stress = None
    if not args.no_stress:
        stress = {}
        for Ps in (workloads.capillary_ratio1000_256(), workloads.droplet_paper_256x512()):
            for prec, coup in ((0, 0), (1, 1)):
                ss = qnsch.Solver(**Ps.create_kwargs(), tol=Ps.tol, stream=stream,
                                  precision=prec, coupled=coup)
                ss.set_fields(Ps.fields())
                for _ in range(min(args.warmup, 2)):
                    ss.step(Ps.dt)
                sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(5)]
                scyc = []
                torch.cuda.synchronize()
                for k in range(5):
                    flush.fill_(float(k))
                    sev[k][0].record(stream)
                    n, res = ss.step(Ps.dt)
                    sev[k][1].record(stream)
                    scyc.append(n)
                torch.cuda.synchronize()
                sms = [a.elapsed_time(b) for a, b in sev]
                stress["%s/%s" % (Ps.name, "mixed_coupled" if prec else "fp64")] = {
                    "value": Ps.cells * 5 / (sum(sms) / 1e3), "unit": UNIT,
                    "ms_per_step": float(np.mean(sms)), "vcycles_per_step": float(np.mean(scyc)),
                    "final_residual": res, "steps": 5, "tol": Ps.tol}
                ss.close()

    # ---- the other workloads of Sec. 8 at their sizes: the capillary wave (64^2,
    # FP64, tol 1e-10) and the Rayleigh-Taylor instability (1024x4096, mixed
    # precision, the paper's smoother)
    paper_workloads = None
    roofline_fp32 = None
    if not args.no_workloads:
        paper_workloads = {}
        # 5 untimed steps first, as for the headline: past the start, where the
        # predictor has its history
        for Pw, prec, nsteps in ((workloads.capillary_64(), 0, 10),
                                 (workloads.rayleigh_taylor_1024x4096(), 1, 5)):
            sw = qnsch.Solver(**Pw.create_kwargs(), tol=Pw.tol, stream=stream, precision=prec,
                              **PATH_OPTIONS[Pw.name])
            sw.set_fields(Pw.fields())
            for _ in range(5):
                sw.step(Pw.dt)
            wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(nsteps)]
            wcyc = []
            torch.cuda.synchronize()
            for k in range(nsteps):
                flush.fill_(float(k))
                wev[k][0].record(stream)
                n, res = sw.step(Pw.dt)
                wev[k][1].record(stream)
                wcyc.append(n)
            torch.cuda.synchronize()
            wms = [a.elapsed_time(b) for a, b in wev]
            wtot = replicas.slowest(sum(wms) / 1e3, dev)
            paper_workloads[Pw.name] = {
                "value": world * Pw.cells * nsteps / wtot, "unit": UNIT,
                "ms_per_step": float(np.mean(wms)), "vcycles_per_step": float(np.mean(wcyc)),
                "precision": "mixed" if prec else "FP64", "steps": nsteps, "tol": Pw.tol,
                "final_residual": res,
                "warmup": 5,
                "options": {k: sw.get_option(k) for k in ("wave_cells32", "wave_rows",
                                                           "vanka_team_max32", "nu1", "nu2",
                                                           "nu_coarse", "predictor")}}
            if prec:  # the FP32 smoothers of the mixed path against HBM
                roofline_fp32 = fp32_smoother_roofline(sw, Pw, stream, flush)
            sw.close()

    # ---- per-step cost on the workload of Sec. 9 (the paper's Table 2: CPU
    # seconds per step of the primitive method, m = 16..256, dt = 16 h^2), FP64
    table2 = None
    if not args.no_table2:
        paper_s, paper_proj_s = paper_table2()
        table2 = {}
        # the projection column starts at m = 32: at m = 16, dt = 1/16 its point
        # smoothers diverge on this workload (the discrete system itself is
        # solvable there: Newton with a direct solve converges)
        for m, sch in [(m, 0) for m in (16, 32, 64, 128, 256)] + [(m, 1) for m in (32, 64, 128, 256)]:
            Pm = workloads.convergence_test(m)
            sm = qnsch.Solver(**Pm.create_kwargs(), tol=Pm.tol, maxcyc=100, stream=stream,
                              scheme=sch)
            sm.set_fields(Pm.fields())
            sm.step(Pm.dt)
            mev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(4)]
            mcyc = []
            torch.cuda.synchronize()
            for k in range(4):
                mev[k][0].record(stream)
                n, _ = sm.step(Pm.dt)
                mev[k][1].record(stream)
                mcyc.append(n)
            torch.cuda.synchronize()
            mms = [a.elapsed_time(b) for a, b in mev]
            table2[("projection/" if sch else "primitive/") + str(m)] = {
                "ms_per_step": float(np.mean(mms)),
                "cell_updates_per_s": m * m / (float(np.mean(mms)) / 1e3),
                "vcycles_per_step": float(np.mean(mcyc)), "tol": Pm.tol,
                "paper_cpu_s_per_step": (paper_proj_s if sch else paper_s)[m]}
            sm.close()

    # ---- batched: the 64-drop workload (grids 64^2 .. 512^2, rho ratio 2..100,
    # viscosity ratio 1..50), mixed precision, coupled smoother, all instances
    # advanced together by qnsch_batch_step
    batched = None
    if not args.no_batch:
        probs = workloads.batch_drops(n=args.batch)
        sols = []
        # options for throughput (serve.THROUGHPUT_OPTIONS): with 64 instances in
        # flight the GPU is full, so one lane per coupled block, larger fused
        # coarse levels and one pre-smoothing step do less work in all
        from paper_1703_06606_gb300 import serve
        bopts = dict(serve.THROUGHPUT_OPTIONS)
        for Pb in probs:
            sb = qnsch.Solver(**Pb.create_kwargs(), tol=Pb.tol, precision=1, coupled=1, **bopts)
            sb.set_fields(Pb.fields())
            sols.append(sb)
        B = qnsch.Batch(sols)
        dts = [Pb.dt for Pb in probs]
        bad = 0
        for _ in range(args.warmup):
            st, _ = B.step(dts)
            bad += sum(1 for x in st if x != 0)
        torch.cuda.synchronize()
        bms, bcyc, spans = [], [], []
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, cy = B.step(dts)
            bms.append((time.perf_counter() - t0) * 1e3)
            spans.append(B.step_times())
            bad += sum(1 for x in st if x != 0)
            bcyc.append(float(np.mean(cy)))
        bcells = sum(Pb.cells for Pb in probs)
        # where the batch step goes: each member's span on its stream inside the
        # batch, and each member's step alone (events on its own stream, one
        # step after the timed ones, the others idle)
        spans = np.concatenate(spans)
        alone = []
        for sb, Pb in zip(sols, probs):
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ea.record(stream)
            sb.set_stream(stream)
            sb.step(Pb.dt)
            eb.record(stream)
            torch.cuda.synchronize()
            alone.append(ea.elapsed_time(eb))
        by_grid = {}
        for Pb, ms in zip(probs, alone):
            by_grid.setdefault("%dx%d" % (Pb.m1, Pb.m2), []).append(ms)
        btot = replicas.slowest(sum(bms) / 1e3, dev)
        batched = {"value": world * bcells * args.steps / btot, "unit": UNIT,
                   "instances": len(probs), "cells": bcells,
                   "ms_per_batch_step": float(np.mean(bms)),
                   "latency_ms": {"p50": float(np.percentile(bms, 50)),
                                  "p99": float(np.percentile(bms, 99))},
                   "mean_vcycles_per_step": float(np.mean(bcyc)), "failed_steps": bad,
                   "precision": "FP32 FAS cycles on the error equation; FP64 residual, "
                                "defect correction, gauge, mass, energy",
                   "smoother": "coupled 7x7 block", "tol": 1e-9, "options": bopts,
                   "timing": "host wall clock per batch step (it synchronises every stream)",
                   "breakdown": {
                       "member_span_ms": {"p50": float(np.percentile(spans, 50)),
                                          "p99": float(np.percentile(spans, 99)),
                                          "max": float(np.max(spans))},
                       "sum_of_steps_alone_ms": float(np.sum(alone)),
                       "steps_alone_ms_by_grid": {g: {"instances": len(v),
                                                      "mean": float(np.mean(v))}
                                                  for g, v in sorted(by_grid.items())},
                       "what": "member_span: from an event before a member's step to one "
                               "after it on the member's stream, inside the batch; alone: "
                               "each member's step by itself after the timed steps"}}
        B.close()
        for sb in sols:
            sb.close()

    # ---- serving: a Poisson stream of capillary-wave and drop requests at the
    # serving workload's parameters (50 requests/s, N log-uniform in [128, 1024],
    # 50 steps each at dt = 1e-4, mixed precision, 150 GB budget), bounded to
    # --serve-requests requests so that the run ends within seconds; every
    # resident request steps as soon as its own previous step is done
    serving = None
    if not args.no_serve:
        from paper_1703_06606_gb300 import serve
        reqs = serve.poisson_requests(args.serve_requests, rate=50.0, n_min=128, n_max=1024,
                                      steps=args.serve_steps, dt=1e-4)
        srv = serve.Server(budget_bytes=150e9, base_options=serve.THROUGHPUT_OPTIONS)
        reqs, _ = srv.run(reqs, device=local_rank)
        serving = serve.summarize(reqs, srv.wall, srv.max_resident, srv.max_backlog)
        serving.update({"arrivals": "Poisson, 50/s", "grid": "N x N, N log-uniform in "
                        "[128, 1024] (multiple of 64)", "steps_per_request": args.serve_steps,
                        "dt": 1e-4, "budget_bytes": 150e9,
                        "precision": "mixed", "smoother": "coupled 7x7 block",
                        "options": dict(serve.THROUGHPUT_OPTIONS),
                        "stepping": "each request's next step is queued as soon as its own "
                                    "previous step is seen finished (qnsch_step_launch / "
                                    "qnsch_step_poll); step latency = launch to completion "
                                    "seen by the server, step_device_ms = CUDA events around "
                                    "the step on its stream"})

    # ---- end to end through the public API with host buffers (pinned): each
    # step's inputs are the committed state and the earlier states the
    # predictor extrapolates from (qnsch_set_history), its output the new state
    def pinned():
        return {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True).numpy()
                for k, v in f0.items()}
    # the same steps as the timed region: from the state and history it started from
    nh = len(start_hist)
    host_in = pinned()
    host_hist = [pinned() for _ in range(nh)]
    for k in host_in:
        host_in[k][...] = start_fields[k]
    for j in range(nh):
        for k in host_in:
            host_hist[j][k][...] = start_hist[j][0][k]
    e2e_ms = []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_fields(host_in)
        for j in range(nh):
            s.set_history(j, host_hist[j], P.dt)
        n, res = s.step(P.dt)
        out = s.get_fields()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        if nh:  # the history moves back by one step on the host
            host_hist.insert(0, host_hist.pop())
            for q in host_in:
                host_hist[0][q][...] = host_in[q]
        for q in host_in:
            host_in[q][...] = out[q]
    e2e_total = replicas.slowest(sum(e2e_ms) / 1e3, dev)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cells = P.cells
    value = world * cells * args.steps / total_s
    e2e_value = world * cells * args.steps / e2e_total
    roofline = roofline_of(kinds, fp64_peak, coarse_smem=s.get_option("coarse_smem_used") == 1)
    step_flops = step_fp64_flops(s, P, float(np.mean(cyc)))
    roofline["step"] = {
        "achieved": step_flops / (float(np.mean(step_ms)) * 1e-3) / 1e12,
        "flops_per_step": step_flops,
        "frac": step_flops / (float(np.mean(step_ms)) * 1e-3) / 1e12 / fp64_peak,
        "what": "algorithmic FP64 operations of a whole step (per-visit counts of the Vanka, "
                "CH and residual kernels over every level, sweep and V-cycle) over ms_per_step"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(P, levels),
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "vcycles_per_step": float(np.mean(cyc)),
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": (1 + nh) * field_bytes(P),
                "d2h_bytes_per_step": field_bytes(P),
                "what": "the timed region's steps again, from the state it started from: per "
                        "step the committed state and the %d earlier states the predictor "
                        "extrapolates from copied in from pinned host memory, one step, the new "
                        "state copied out" % nh},
        "gpu_launches": int(launches),
        "device_loop": bool(device_loop),
        "roofline": roofline,
        "kernel_shares": {k: {kk: v[kk] for kk in ("launches", "ms_per_step", "share", "visits")}
                          for k, v in kinds["kinds"].items()},
        "clocks": clk.summary(),
    }
    if variants:
        line["variants"] = variants
    if stress is not None:
        line["stress"] = stress
    if paper_workloads is not None:
        line["workloads"] = paper_workloads
    if roofline_fp32 is not None:
        line["roofline_fp32"] = roofline_fp32
    if table2 is not None:
        line["table2"] = table2
    if batched is not None:
        line["batched"] = batched
    if serving is not None:
        line["serving"] = serving
    if world == 1 and not args.no_cpu_baseline:
        times, cycles = oracle_rate(P, steps=3, budget_s=args.cpu_budget, fields=start_fields,
                                    options=PATH_OPTIONS["fp64"], history=start_hist)
        line["cpu_baseline"] = {
            "value": cells * len(times) / sum(times), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "time steps %d..%d of the rising-droplet 256x512 workload (the first %d "
                      "of the GPU's timed steps, from the GPU's committed state after its %d "
                      "warm-up steps), serial FP64 oracle, %.1f s"
                      % (args.warmup + 1, args.warmup + len(times), len(times), args.warmup,
                         sum(times)),
            "vcycles": cycles, "gpu_vcycles_same_steps": cyc[:len(times)],
            "options": dict(PATH_OPTIONS["fp64"])}
        line["cpu_baseline"]["host"] = host_cpu()
        if not args.no_cpu_all_cores:
            line["cpu_baseline"]["all_cores"] = oracle_all_cores(steps=1,
                                                                 options=PATH_OPTIONS["fp64"])
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# algorithmic FP64 operations per Vanka cell visit (add/sub/mul/div = 1, fused
# multiply-add = 2), counted from the formulas of one 5x5 Vanka block (Sec. 7.1)
# as the kernel evaluates it: 4 edge averages of the densities rho(c) (read from
# the array the smoothers keep), 4 diagonals from the per-step row
# coefficients, off-diagonals and the mass row, 4 momentum residuals from the
# per-step assembled stencils and 1 mass residual, the structured block solve,
# 5 updates
VANKA_FP64_FLOPS_PER_VISIT = 287.0
# FP64 operations per CH cell visit (N_c, N_mu, the 2x2 Jacobian, its solve and
# rho of the new c) and per residual cell (all five families), as ncu counts
# them executed (add, mul = 1, fma = 2) on the FP64 kernels
CH_FP64_FLOPS_PER_VISIT = 241.0
RESIDUAL_FP64_FLOPS_PER_CELL = 223.0
# dram__bytes_read.sum + dram__bytes_write.sum per launch of a timed kind (average
# over its launches), from one ncu capture of the same kernel build (the
# profiles/ file named beside it; cold-cache, serialised); a kind without a
# capture of the current build reports traffic null.  Drop these entries when
# the kernels change.
TRAFFIC_BYTES = {
    "vanka_levels": (3.08e6, "profiles/dram_per_kernel_fp64_step_rising_drop_256x512.md"),
    "vanka_finest": (33.99e6, "profiles/dram_per_kernel_fp64_step_rising_drop_256x512.md"),
    "coarse_vcycle": (0.39e6, "profiles/dram_per_kernel_fp64_step_rising_drop_256x512.md"),
    "ch": (15.66e6, "profiles/dram_per_kernel_fp64_step_rising_drop_256x512.md"),
    "vanka_finest_fp32": (431.99e6, "profiles/dram_per_kernel_rayleigh_taylor_1024x4096.md"),
    "ch_fp32": (299.10e6, "profiles/dram_per_kernel_rayleigh_taylor_1024x4096.md"),
}
# words per cell a sweep moves at one pass over the arrays it needs (Sec. 7.1
# smoothers; read c^n, u^n, v^n, c, mu, u, v, p and the three right-hand sides,
# write u, v, p for the Vanka block; c^n, u, v, c, mu, p and two right-hand
# sides, write c, mu for the CH block)
VANKA_WORDS_PER_CELL = 14
CH_WORDS_PER_CELL = 10


def prof_kinds(s, P, stream, flush, nsteps):
    """Time each kind of launch (qnsch_profile's kinds) with CUDA events over
    `nsteps` steps of the workload, and the steps themselves; per kind: launches,
    ms per step, share of the step's device time, cell visits per step."""
    import torch
    s.profile(15)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(nsteps)]
    cyc = []
    for k in range(nsteps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        n, _ = s.step(P.dt)
        ev[k][1].record(stream)
        cyc.append(n)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    out = {"steps": nsteps, "ms_per_step": float(np.mean(ms)), "vcycles": cyc, "kinds": {}}
    for kind in s.PROFILE_KINDS:
        n, tot, vis = s.profile_read_kind(kind)
        out["kinds"][kind] = {"launches": n, "ms_per_step": tot / nsteps,
                              "share": tot / max(sum(ms), 1e-30), "visits": vis / nsteps,
                              "avg_launch_us": 1e3 * tot / max(n, 1),
                              "visits_per_launch": vis / max(n, 1)}
    s.profile(False)
    return out


def hbm_peak_gbs():
    """The measured HBM copy bandwidth of this machine's GPUs (MEASURED_PEAKS.json
    beside this file), else the earlier measurement of 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback (6.8 TB/s, an earlier GB300 measurement)"


def fp32_smoother_roofline(s, P, stream, flush, nsteps=2):
    """The FP32 smoothers of the mixed path on a large workload, against HBM:
    algorithmic bytes (one pass over the words a sweep needs, VANKA_WORDS_PER_CELL
    and CH_WORDS_PER_CELL in FP32) over the event-timed duration of the finest
    level's smoothing launches.  With the banded wavefront (wave_cells32) one
    launch runs nu smoothing steps of both smoothers; without it the finest
    level's Vanka colour launches and CH colour launches are timed apart."""
    import torch
    hbm, src = hbm_peak_gbs()
    s.profile(1 | 8 | 16)
    for k in range(nsteps):
        flush.fill_(float(k))
        s.step(P.dt)
    torch.cuda.synchronize()
    out = {"workload": P.name, "peak": hbm, "unit": "GB/s", "peak_source": src,
           "bound": "hbm", "kernels": {}}
    per_cell = {"wave": 4 * (VANKA_WORDS_PER_CELL + CH_WORDS_PER_CELL),
                "vanka_finest": 4 * VANKA_WORDS_PER_CELL, "ch": 4 * CH_WORDS_PER_CELL}
    for kind in ("wave", "vanka_finest", "ch"):
        n, ms, vis = s.profile_read_kind(kind)
        if n == 0:
            continue
        gbs = vis * per_cell[kind] / (ms * 1e-3) / 1e9
        tr = TRAFFIC_BYTES.get(kind + "_fp32")
        out["kernels"][kind] = {"launches": n, "avg_launch_us": 1e3 * ms / n,
                                "visits_per_launch": vis / n,
                                "algorithmic_bytes_per_launch": vis / n * per_cell[kind],
                                "achieved": gbs, "frac": gbs / hbm,
                                "traffic": tr[0] if tr else None,
                                "traffic_source": tr[1] if tr else None}
    s.profile(False)
    return out


def roofline_of(kinds, fp64_peak, coarse_smem=False):
    """The roofline entry of the dominant kind of launch (largest share of the
    step's device time): algorithmic FP64 operations per launch over its
    average event-timed duration, against the FP64 peak measured in this run.
    coarse_smem: the fused coarse V-cycle ran on its shared-memory copy."""
    name, k = max(kinds["kinds"].items(), key=lambda kv: kv[1]["share"])
    per_visit = {"vanka_finest": VANKA_FP64_FLOPS_PER_VISIT,
                 "vanka_levels": VANKA_FP64_FLOPS_PER_VISIT,
                 "coarse_vcycle": VANKA_FP64_FLOPS_PER_VISIT + CH_FP64_FLOPS_PER_VISIT,
                 "ch": CH_FP64_FLOPS_PER_VISIT}[name]
    flops = k["visits_per_launch"] * per_visit
    achieved = flops / (k["avg_launch_us"] * 1e-6) / 1e12
    kernel = {"vanka_finest": "k_vanka<double> (finest level)",
              "vanka_levels": "k_vanka_team<double> (levels below the finest)",
              "coarse_vcycle": ("k_coarse_vcycle_smem (fused coarse levels, shared-memory copy)"
                                if coarse_smem else "k_coarse_vcycle<double> (fused coarse levels)"),
              "ch": "k_ch<double> (finest level)"}[name]
    tr = TRAFFIC_BYTES.get(name)
    return {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
            "frac": achieved / fp64_peak, "traffic": tr[0] if tr else None,
            "traffic_source": tr[1] if tr else None,
            "kernel": kernel, "share_of_step": k["share"], "launches_timed": k["launches"],
            "avg_launch_us": k["avg_launch_us"], "flops_per_launch": flops,
            "peak_source": "qnsch_fma_probe (FP64 FMA throughput, 8 independent chains per "
                           "thread, best of 4/8/16 blocks per SM), run in this process",
            "other_kinds": {n: {"share_of_step": v["share"],
                                "avg_launch_us": v["avg_launch_us"]}
                            for n, v in kinds["kinds"].items() if n != name}}


def step_fp64_flops(s, P, cycles):
    """Algorithmic FP64 operations of one step of `cycles` V-cycles: per V-cycle
    on every level (m1/2^l x m2/2^l cells) nu1 + nu2 smoothing steps
    (nu1_fine + nu2_fine on the finest level when set; one Vanka and one CH
    visit per cell each; the coarsest level nu_coarse ceil(n/4)^2 of them),
    one residual per level above the coarsest and one
    coarse-operator evaluation per level below the finest; per step one
    residual of the initial state and one per V-cycle with the norms."""
    nlev = s.levels
    nu = s.get_option("nu1") + s.get_option("nu2")
    n1f, n2f = s.get_option("nu1_fine"), s.get_option("nu2_fine")
    nu0 = (n1f if n1f >= 0 else s.get_option("nu1")) + (n2f if n2f >= 0 else s.get_option("nu2"))
    nuc = s.get_option("nu_coarse")
    smooth = VANKA_FP64_FLOPS_PER_VISIT + CH_FP64_FLOPS_PER_VISIT
    per_cycle = 0.0
    for l in range(nlev):
        c = (P.m1 >> l) * (P.m2 >> l)
        if l == nlev - 1:
            n = max(P.m1 >> l, P.m2 >> l)
            q = max(1, (n + 3) // 4)
            per_cycle += nuc * q * q * c * smooth
        else:
            per_cycle += (nu0 if l == 0 else nu) * c * smooth + c * RESIDUAL_FP64_FLOPS_PER_CELL
        if l > 0:
            per_cycle += c * RESIDUAL_FP64_FLOPS_PER_CELL
    per_cycle += P.cells * RESIDUAL_FP64_FLOPS_PER_CELL  # the norms' residual
    return cycles * per_cycle + P.cells * RESIDUAL_FP64_FLOPS_PER_CELL


def run_reference(args, rank, world):
    if rank != 0:
        return
    P = workloads.rising_drop_256x512()
    per_step_budget = 150.0 / max(args.steps + args.warmup, 1)
    # warm-up: one short untimed oracle call on a small case
    from oracle.ref import RefSolver
    w = workloads.small_case(32, 32, False)
    r = RefSolver(**w.create_kwargs())
    r.set_fields(w.fields())
    for _ in range(min(args.warmup, 3)):
        r.step(w.dt)
    times, cycles = oracle_rate(P, steps=args.steps, budget_s=max(per_step_budget * args.steps, 20.0),
                                options=PATH_OPTIONS["fp64"])
    value = P.cells * len(times) / sum(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": len(times),
        "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(P, 8), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "host": host_cpu(),
                         "sample": "first %d time step(s) of the workload from its initial "
                                   "state (%s V-cycles)" % (len(times),
                                                            "/".join(map(str, cycles)))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-stress", action="store_true")
    ap.add_argument("--no-workloads", action="store_true")
    ap.add_argument("--no-table2", action="store_true")
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-steps", type=int, default=50)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
