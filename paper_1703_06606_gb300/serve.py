"""Continuous-batching server for independent q-NSCH simulations.

Requests (a workload and a number of time steps) arrive over time.  An
admission thread takes them in arrival order, and as soon as a slot is free and
a request's device footprint (qnsch_footprint) fits the memory budget it
creates the simulation (fields and multigrid hierarchy resident on the GPU,
off the stepping loop's critical path).  The stepping loop advances every
resident simulation independently: each one's next time step is queued
(qnsch_step_launch, one graph on its own stream) the moment its previous step
is seen finished, and each of its outer cycles as soon as the previous
cycle's norms are seen (qnsch_step_poll drives the host-driven loop), so the
simulations' kernels overlap on the device and a small simulation never waits
for a large one.  A simulation
leaves when it has done its steps (or failed), which frees its memory for the
next request.  Each simulation goes through exactly the arithmetic it would
alone, so its result does not depend on the mix.  Per step the server records
the wall time from launch to completion seen by the loop and the step's device
time (CUDA events around it on the simulation's stream).

    python -m paper_1703_06606_gb300.serve --requests 40 --rate 50 --steps 20
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import json
import math
import threading
import time

import numpy as np

from . import autotune, qnsch, workloads

# Options for many simulations in flight at once (mixed precision, coupled
# block), where the GPU is full and work, not one simulation's latency,
# decides.  One lane per coupled block in the per-level launches: the
# four-lane teams repeat part of each visit on every lane.  Levels up to 2048
# cells go into each simulation's single-block V-cycle, which holds one SM.
# One smoothing step before the coarse-grid correction and two after it: more
# V-cycles per time step, fewer smoothing visits in all.  Measured on the
# 64-drop batch, in ms per batch step: 114.2 with (nu1, nu2) = (2, 2); 101.6
# with (1, 2); 111.6 with (1, 1); 111.7 with (2, 1); 107.9 with (1, 3).  Each
# step starting from the quadratic extrapolation in time of the last three
# states (predictor 2): 83.2 against 98.7 without and 89.3 with the linear
# one (after 5 warm-up steps).  The FP64 defect correction still decides the
# answer at the same tolerance.
THROUGHPUT_OPTIONS = {"fuse_cells32": 2048, "vanka_team_max32": 0, "nu1": 1, "nu2": 2,
                      "predictor": 2}


@dataclasses.dataclass
class Request:
    rid: int
    problem: workloads.Problem
    steps: int
    arrival: float          # seconds after the start of the run
    admitted: float = math.nan
    finished: float = math.nan
    done_steps: int = 0
    status: int = 0
    step_ms: list = dataclasses.field(default_factory=list)
    device_ms: list = dataclasses.field(default_factory=list)
    vcycles: list = dataclasses.field(default_factory=list)


def poisson_requests(n, rate, seed=workloads.SEED, n_min=128, n_max=1024, steps=50, dt=1e-4):
    """n requests with exponential inter-arrival times of mean 1/rate: half
    capillary waves, half rising drops, square grids N x N with N log-uniform in
    [n_min, n_max] rounded to a multiple of 64."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n):
        t += rng.exponential(1.0 / rate)
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) / 64.0)) * 64
        N = max(64, N)
        if rng.random() < 0.5:
            P = workloads.capillary_64()
            P.m1 = P.m2 = N
            P.Cn = 0.01
        else:
            P = workloads.batch_drops(n=1, seed=int(rng.integers(1 << 30)))[0]
            P.m1 = P.m2 = N
            P.Cn = 2.5 / N
            P.Pe = 1.0 / P.Cn
            P.init_args = dict(P.init_args, y0=0.5)
        P.name = "req%d_%s_%d" % (k, "capillary" if P.init == "capillary" else "drop", N)
        P.dt = dt
        P.tol = 1e-9
        out.append(Request(k, P, steps, t))
    return out


class Server:
    def __init__(self, budget_bytes=150e9, max_slots=256, precision=1, coupled=1,
                 tuned_table=None, backend=None, base_options=None):
        """tuned_table: an autotune table (dict, or the path of its JSON file)
        whose entries give the launch-shape options of matching requests.
        base_options: solver options for every simulation (for example
        THROUGHPUT_OPTIONS); a matching tuned-table entry overrides them.
        backend: the module that provides Solver, Batch and footprint (the
        qnsch binding; another object with the same three names drives the
        admission and batching logic without a GPU)."""
        self.qn = backend or qnsch
        self.budget = budget_bytes
        self.max_slots = max_slots
        self.precision = precision
        self.coupled = coupled
        if isinstance(tuned_table, str):
            tuned_table = autotune.load_table(tuned_table)
        self.tuned = tuned_table or {}
        self.device = autotune.device_name() if self.tuned else ""
        self.base_options = dict(base_options or {})

    def options(self, P):
        """Options of a request: the base options, then the tuned table's
        entry for it (if any) on top."""
        out = dict(self.base_options)
        if self.tuned:
            out.update(autotune.lookup(self.tuned, P, self.precision, self.coupled, 0,
                                       self.device))
        return out

    def footprint(self, P):
        return self.qn.footprint(P.m1, P.m2, P.periodic_x, P.levels, self.precision, P.Lx)

    def run(self, requests, keep_fields=False, device=None, poll_sleep_s=20e-6):
        """Serve `requests` (arrival times relative to now) to completion; returns
        the requests (with timings) and, if keep_fields, their final fields.
        device: the CUDA device index the admission thread makes current before
        it creates simulations (None: the thread's default)."""
        waiting = collections.deque(sorted(requests, key=lambda r: r.arrival))
        ready = collections.deque()  # admitted (request, solver, footprint)
        cond = threading.Condition()
        state = {"used": 0, "slots": 0, "admitting": True, "error": None, "max_wait": 0,
                 "max_used": 0}
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731

        def admit():
            try:
                if device is not None:
                    import torch
                    torch.cuda.set_device(device)
                while waiting:
                    r = waiting[0]
                    delay = r.arrival - clock()
                    if delay > 0:
                        time.sleep(delay)
                    fp = self.footprint(r.problem)
                    if fp > self.budget:
                        raise ValueError("request %d needs %d bytes, more than the budget"
                                         % (r.rid, fp))
                    with cond:
                        # first in line waits for memory and a slot
                        while (state["used"] + fp > self.budget or
                               state["slots"] >= self.max_slots):
                            cond.wait()
                        state["used"] += fp
                        state["slots"] += 1
                        state["max_used"] = max(state["max_used"], state["used"])
                    waiting.popleft()
                    P = r.problem
                    # host-driven steps: many resident simulations' whole-step
                    # graphs (device_loop) measured slower than their cycles
                    # queued from the host as each one's norms arrive
                    sv = self.qn.Solver(**P.create_kwargs(), tol=P.tol, precision=self.precision,
                                        coupled=self.coupled, device_loop=0,
                                        **self.options(P))
                    sv.set_fields(P.fields())
                    r.admitted = clock()
                    with cond:
                        ready.append((r, sv, fp))
                        backlog = sum(1 for w in waiting if w.arrival <= clock())
                        state["max_wait"] = max(state["max_wait"], backlog)
            except BaseException as e:  # noqa: BLE001 - reported by the stepping loop
                state["error"] = e
            finally:
                with cond:
                    state["admitting"] = False

        th = threading.Thread(target=admit, daemon=True)
        th.start()
        inflight = []  # [request, solver, footprint, launch time]
        fields = {}
        max_res = 0
        try:
            while True:
                with cond:
                    new = list(ready)
                    ready.clear()
                    admitting = state["admitting"]
                for r, sv, fp in new:
                    sv.step_launch(r.problem.dt)
                    inflight.append([r, sv, fp, clock()])
                max_res = max(max_res, len(inflight))
                if not inflight:
                    if state["error"] is not None:
                        raise state["error"]
                    if not admitting:
                        with cond:
                            if not ready:
                                break
                        continue
                    time.sleep(poll_sleep_s)
                    continue
                progressed = False
                keep = []
                for item in inflight:
                    r, sv, fp, tl = item
                    out = sv.step_poll()
                    if out is None:
                        keep.append(item)
                        continue
                    progressed = True
                    now = clock()
                    nc, _, code, dms = out
                    r.step_ms.append(1e3 * (now - tl))
                    r.device_ms.append(dms)
                    r.vcycles.append(nc)
                    r.done_steps += 1
                    if code != 0:
                        r.status = code
                    if code != 0 or r.done_steps >= r.steps:
                        r.finished = now
                        if keep_fields:
                            fields[r.rid] = sv.get_fields()
                        sv.close()
                        with cond:
                            state["used"] -= fp
                            state["slots"] -= 1
                            cond.notify_all()
                    else:
                        sv.step_launch(r.problem.dt)
                        item[3] = clock()
                        keep.append(item)
                inflight = keep
                if not progressed:
                    time.sleep(poll_sleep_s)
        finally:
            th.join(timeout=60)
        if state["error"] is not None:
            raise state["error"]
        self.max_resident = max_res
        self.max_backlog = state["max_wait"]
        self.max_used_bytes = state["max_used"]
        self.wall = clock()
        return requests, fields


def summarize(reqs, wall, max_resident, max_backlog=None):
    """Throughput and latency of a served stream.  offered_cell_steps_per_s is
    the work the arrivals asked for per second of the arrival span; when the
    server delivers well below it the queue grows for the whole run
    (saturated)."""
    steps = [ms for r in reqs for ms in r.step_ms]
    dev = [ms for r in reqs for ms in r.device_ms if ms >= 0]
    lat = [1e3 * (r.finished - r.arrival) for r in reqs]
    wait = [1e3 * (r.admitted - r.arrival) for r in reqs]
    cell_steps = sum(r.problem.cells * r.done_steps for r in reqs)
    span = max(r.arrival for r in reqs) - min(r.arrival for r in reqs)
    offered = sum(r.problem.cells * r.steps for r in reqs) / span if span > 0 else math.inf
    value = cell_steps / wall
    out = {"value": value, "unit": "cell-updates/s", "requests": len(reqs),
           "failed": sum(1 for r in reqs if r.status != 0), "wall_s": wall,
           "cell_steps": cell_steps, "max_resident": max_resident,
           "offered_cell_steps_per_s": offered, "saturated": bool(value < 0.9 * offered),
           "step_latency_ms": {"p50": float(np.percentile(steps, 50)),
                               "p99": float(np.percentile(steps, 99))},
           "request_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                  "p99": float(np.percentile(lat, 99))},
           "queue_wait_ms": {"p50": float(np.percentile(wait, 50)),
                             "p99": float(np.percentile(wait, 99))},
           "mean_vcycles_per_step": float(np.mean([c for r in reqs for c in r.vcycles]))}
    if dev:
        out["step_device_ms"] = {"p50": float(np.percentile(dev, 50)),
                                 "p99": float(np.percentile(dev, 99))}
    if max_backlog is not None:
        out["max_backlog"] = max_backlog
    return out


def request_record(r):
    """One request's log line: its grid and steps, arrival, admission and
    finish times (seconds from the start of the run), per-step latencies (ms),
    V-cycles per step and final status."""
    return {"request": r.rid, "workload": r.problem.name, "grid": [r.problem.m1, r.problem.m2],
            "steps": r.steps, "done_steps": r.done_steps, "status": r.status,
            "arrival_s": r.arrival, "admitted_s": r.admitted, "finished_s": r.finished,
            "queue_wait_ms": 1e3 * (r.admitted - r.arrival),
            "latency_ms": 1e3 * (r.finished - r.arrival),
            "step_ms": list(r.step_ms), "device_ms": list(r.device_ms),
            "vcycles": list(r.vcycles)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--nmin", type=int, default=128)
    ap.add_argument("--nmax", type=int, default=1024)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--log", default=None, help="JSON lines, one per request")
    ap.add_argument("--defaults", action="store_true",
                    help="the library's single-instance defaults instead of THROUGHPUT_OPTIONS")
    a = ap.parse_args()
    reqs = poisson_requests(a.requests, a.rate, n_min=a.nmin, n_max=a.nmax, steps=a.steps)
    srv = Server(budget_bytes=a.budget_gb * 1e9,
                 base_options=None if a.defaults else THROUGHPUT_OPTIONS)
    reqs, _ = srv.run(reqs)
    if a.log:
        with open(a.log, "w") as f:
            for r in reqs:
                f.write(json.dumps(request_record(r)) + "\n")
    print(json.dumps(summarize(reqs, srv.wall, srv.max_resident, srv.max_backlog)))


if __name__ == "__main__":
    main()
