"""Continuous-batching server for independent q-NSCH simulations.

Requests (a workload and a number of time steps) arrive over time.  The server
keeps every admitted simulation's fields and multigrid hierarchy resident on
the GPU, admits waiting requests in arrival order as soon as a slot is free and
their device footprint (qnsch_footprint) fits the memory budget, and advances
all resident simulations together, one time step per round, through
qnsch_batch_step (their kernels overlap on the device).  A simulation leaves
when it has done its steps (or failed).  Each simulation goes through exactly
the arithmetic it would alone, so its result does not depend on the mix.

    python -m paper_1703_06606_gb300.serve --requests 40 --rate 50 --steps 20
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import time

import numpy as np

from . import autotune, qnsch, workloads


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
                 tuned_table=None, backend=None):
        """tuned_table: an autotune table (dict, or the path of its JSON file)
        whose entries give the launch-shape options of matching requests.
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

    def options(self, P):
        """Launch-shape options of a request from the tuned table ({} if none)."""
        if not self.tuned:
            return {}
        return autotune.lookup(self.tuned, P, self.precision, self.coupled, 0, self.device)

    def footprint(self, P):
        return self.qn.footprint(P.m1, P.m2, P.periodic_x, P.levels, self.precision, P.Lx)

    def run(self, requests, keep_fields=False):
        """Serve `requests` (arrival times relative to now) to completion; returns
        the requests (with timings) and, if keep_fields, their final fields."""
        waiting = sorted(requests, key=lambda r: r.arrival)
        resident = []  # (request, solver, footprint)
        used = 0
        t0 = time.perf_counter()
        fields = {}
        max_res = 0
        while waiting or resident:
            now = time.perf_counter() - t0
            while (waiting and waiting[0].arrival <= now and len(resident) < self.max_slots):
                r = waiting[0]
                fp = self.footprint(r.problem)
                if fp > self.budget:
                    raise ValueError("request %d needs %d bytes, more than the budget"
                                     % (r.rid, fp))
                if used + fp > self.budget:
                    break  # first in line waits for memory
                waiting.pop(0)
                P = r.problem
                s = self.qn.Solver(**P.create_kwargs(), tol=P.tol, precision=self.precision,
                                   coupled=self.coupled, **self.options(P))
                s.set_fields(P.fields())
                r.admitted = time.perf_counter() - t0
                resident.append((r, s, fp))
                used += fp
            max_res = max(max_res, len(resident))
            if not resident:
                time.sleep(max(0.0, waiting[0].arrival - (time.perf_counter() - t0)))
                continue
            B = self.qn.Batch([s for _, s, _ in resident])
            ts = time.perf_counter()
            st, cyc = B.step([r.problem.dt for r, _, _ in resident])
            dur = (time.perf_counter() - ts) * 1e3
            B.close()
            keep = []
            for (r, s, fp), code, nc in zip(resident, st, cyc):
                r.step_ms.append(dur)
                r.vcycles.append(nc)
                r.done_steps += 1
                if code != 0:
                    r.status = code
                if code != 0 or r.done_steps >= r.steps:
                    r.finished = time.perf_counter() - t0
                    if keep_fields:
                        fields[r.rid] = s.get_fields()
                    s.close()
                    used -= fp
                else:
                    keep.append((r, s, fp))
            resident = keep
        self.max_resident = max_res
        self.wall = time.perf_counter() - t0
        return requests, fields


def summarize(reqs, wall, max_resident):
    steps = [ms for r in reqs for ms in r.step_ms]
    lat = [1e3 * (r.finished - r.arrival) for r in reqs]
    wait = [1e3 * (r.admitted - r.arrival) for r in reqs]
    cell_steps = sum(r.problem.cells * r.done_steps for r in reqs)
    return {"value": cell_steps / wall, "unit": "cell-updates/s", "requests": len(reqs),
            "failed": sum(1 for r in reqs if r.status != 0), "wall_s": wall,
            "cell_steps": cell_steps, "max_resident": max_resident,
            "step_latency_ms": {"p50": float(np.percentile(steps, 50)),
                                "p99": float(np.percentile(steps, 99))},
            "request_latency_ms": {"p50": float(np.percentile(lat, 50)),
                                   "p99": float(np.percentile(lat, 99))},
            "queue_wait_ms": {"p50": float(np.percentile(wait, 50)),
                              "p99": float(np.percentile(wait, 99))},
            "mean_vcycles_per_step": float(np.mean([c for r in reqs for c in r.vcycles]))}


def request_record(r):
    """One request's log line: its grid and steps, arrival, admission and
    finish times (seconds from the start of the run), per-step latencies (ms),
    V-cycles per step and final status."""
    return {"request": r.rid, "workload": r.problem.name, "grid": [r.problem.m1, r.problem.m2],
            "steps": r.steps, "done_steps": r.done_steps, "status": r.status,
            "arrival_s": r.arrival, "admitted_s": r.admitted, "finished_s": r.finished,
            "queue_wait_ms": 1e3 * (r.admitted - r.arrival),
            "latency_ms": 1e3 * (r.finished - r.arrival),
            "step_ms": list(r.step_ms), "vcycles": list(r.vcycles)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=40)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--nmin", type=int, default=128)
    ap.add_argument("--nmax", type=int, default=1024)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--log", default=None, help="JSON lines, one per request")
    a = ap.parse_args()
    reqs = poisson_requests(a.requests, a.rate, n_min=a.nmin, n_max=a.nmax, steps=a.steps)
    srv = Server(budget_bytes=a.budget_gb * 1e9)
    reqs, _ = srv.run(reqs)
    if a.log:
        with open(a.log, "w") as f:
            for r in reqs:
                f.write(json.dumps(request_record(r)) + "\n")
    print(json.dumps(summarize(reqs, srv.wall, srv.max_resident)))


if __name__ == "__main__":
    main()
